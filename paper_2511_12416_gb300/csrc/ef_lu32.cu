// FP32 minors of the Exact algorithm (Eq. 3 for every (pattern, bitstring) of
// a mode block), one thread per bitstring, the minor in registers: the single
// circuit kernel and the work-queue kernel of multi-circuit batches. Kept in a
// translation unit of their own so that the library's sources compile in
// parallel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ef_common.cuh"
#include "ef_internal.h"

namespace ef {

// ---------------------------------------------------------------- 2a. FP32, thread per minor
// Thread <-> bitstring; the CTA stages one chunk of 2^c_log2 pattern matrices
// (row stride ETA|1 float2 so that the rows of a matrix fall in distinct
// banks) and every thread factors its own minor of each, in registers.

int exact_f32_chunk_log2(int n, int eta, int r, int64_t nb) {
    int cl = std::min(r, 5);
    while (cl > 0 && ((size_t)1 << cl) * n * (size_t)(eta | 1) * sizeof(float2) > 48 * 1024) --cl;
    // keep at least ~5 waves of 3 CTAs per SM (measured on the 32-qubit workload:
    // 8 patterns per chunk beat 4 by 2 % and 16 lose 5 %)
    const int64_t tiles = (nb + 127) / 128;
    while (cl > 0 && tiles * ((int64_t)1 << (r - cl)) < (int64_t)sm_count() * 3 * 5) --cl;
    return cl;
}

template <int ETA>
__global__ void __launch_bounds__(128) k_exact_lu_f32(ExactBlockDev B0, ExactBlockDev B1,
                                                      const uint64_t* __restrict__ bits, int64_t nb) {
    cudaGridDependencySynchronize();  // see launch_pdl
    extern __shared__ float2 smM[];
    // both mode blocks in one launch (blockIdx.z): one tail instead of two
    const ExactBlockDev& B = blockIdx.z ? B1 : B0;
    constexpr int S = ETA | 1;
    const int n = B.n;
    const int Y = 1 << B.c_log2;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int rows[ETA];
    const bool ok = (b < nb) && decode_rows<ETA>(bits[2 * b], bits[2 * b + 1], B.mask0, B.mask1, rows);
    for (int chunk = blockIdx.y; chunk < B.n_chunks; chunk += gridDim.y) {
        const float2* src = B.M32 + (size_t)chunk * Y * n * ETA;
        __syncthreads();
        for (int e = threadIdx.x; e < Y * n * ETA; e += blockDim.x) {
            const int row = e / ETA, j = e - row * ETA;
            smM[row * S + j] = src[e];
        }
        __syncthreads();
        if (b >= nb) continue;
        // error terms of four consecutive patterns go out as one 8-byte store
        // (chunks of at least 4 patterns start at a multiple of 4)
        const bool pack = Y >= 4;
        uint64_t codes = 0;
        for (int t = 0; t < Y; ++t) {
            const size_t z = (size_t)chunk * Y + t;
            float2 det = make_float2(0.f, 0.f);
            uint16_t ec = 0;
            if (ok) {
                const float2* Mt = smM + (size_t)t * n * S;
                float2 A[ETA][ETA];
#pragma unroll
                for (int i = 0; i < ETA; ++i) {
                    const float2* rp = Mt + rows[i] * S;
#pragma unroll
                    for (int j = 0; j < ETA; ++j) A[i][j] = rp[j];
                }
                float er2, zabs2;
                det = lu_det_regs<float, ETA>(A, er2, zabs2);
                ec = err_term_code(det, er2, zabs2);
            }
            const size_t o = dix(b, (uint32_t)z, B.r);
            B.D32[o] = det;
            if (!pack) {
                B.E32[o] = ec;
            } else {
                codes = (codes >> 16) | ((uint64_t)ec << 48);
                if ((t & 3) == 3) *reinterpret_cast<uint64_t*>(B.E32 + o - 3) = codes;
            }
        }
    }
}

template <int ETA>
static cudaError_t launch_f32_eta(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk, const uint64_t* bits,
                                  int64_t nb, cudaStream_t s) {
    constexpr int S = ETA | 1;
    size_t smem = 0;
    int chunks = 1;
    for (int i = 0; i < nblk; ++i) {
        const ExactBlockDev& b = i ? b1 : b0;
        smem = std::max(smem, (size_t)(1 << b.c_log2) * b.n * S * sizeof(float2));
        chunks = std::max(chunks, b.n_chunks);
    }
    cudaError_t e = raise_dynamic_smem((const void*)k_exact_lu_f32<ETA>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((nb + 127) / 128), (unsigned)std::min(chunks, 65535), (unsigned)nblk);
    e = launch_pdl(k_exact_lu_f32<ETA>, grid, dim3(128), smem, s, b0, nblk == 2 ? b1 : b0, bits, nb);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_exact_lu_f32(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk, const uint64_t* bits,
                                int64_t nb, cudaStream_t s, LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    if (nblk < 1 || nblk > 2 || (nblk == 2 && b1.eta != b0.eta)) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (b0.eta) {
        case 1: e = launch_f32_eta<1>(b0, b1, nblk, bits, nb, s); break;
        case 2: e = launch_f32_eta<2>(b0, b1, nblk, bits, nb, s); break;
        case 3: e = launch_f32_eta<3>(b0, b1, nblk, bits, nb, s); break;
        case 4: e = launch_f32_eta<4>(b0, b1, nblk, bits, nb, s); break;
        case 5: e = launch_f32_eta<5>(b0, b1, nblk, bits, nb, s); break;
        case 6: e = launch_f32_eta<6>(b0, b1, nblk, bits, nb, s); break;
        case 7: e = launch_f32_eta<7>(b0, b1, nblk, bits, nb, s); break;
        case 8: e = launch_f32_eta<8>(b0, b1, nblk, bits, nb, s); break;
        case 9: e = launch_f32_eta<9>(b0, b1, nblk, bits, nb, s); break;
        case 10: e = launch_f32_eta<10>(b0, b1, nblk, bits, nb, s); break;
        default: return cudaErrorInvalidValue;
    }
    st.launches += 1;
    for (int i = 0; i < nblk; ++i) st.executed_lus += nb * ((int64_t)1 << (i ? b1 : b0).r);
    return e;
}

// ---------------------------------------------------------------- 2a'. FP32 work queue over several circuits
// Persistent kernel for a batch of circuits whose blocks share eta: every CTA
// repeatedly takes the next (circuit block, bitstring tile, pattern chunk)
// item from a device counter, stages that chunk's matrices and factors the
// minors of its 128 bitstrings exactly as k_exact_lu_f32 does. CTAs leave
// when the queue is empty (no CTA ever waits for another).

template <int ETA>
__global__ void __launch_bounds__(128) k_queue_lu_f32(const QueueEntry* __restrict__ q, int nq, int64_t n_items,
                                                      unsigned long long* __restrict__ head) {
    extern __shared__ float2 smQ[];
    __shared__ long long s_item;
    constexpr int S = ETA | 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(head, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        int lo = 0, hi = nq - 1;  // last entry with item_begin <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (q[mid].item_begin <= item) lo = mid;
            else hi = mid - 1;
        }
        const QueueEntry& E = q[lo];
        const ExactBlockDev& B = E.blk;
        const int64_t local = item - E.item_begin;
        const int chunk = (int)(local / E.tiles);
        const int64_t tile = local - (int64_t)chunk * E.tiles;
        const int n = B.n;
        const int Y = 1 << B.c_log2;
        const float2* src = B.M32 + (size_t)chunk * Y * n * ETA;
        for (int e = threadIdx.x; e < Y * n * ETA; e += blockDim.x) {
            const int row = e / ETA, j = e - row * ETA;
            smQ[row * S + j] = src[e];
        }
        __syncthreads();
        const int64_t b = tile * 128 + threadIdx.x;
        if (b < E.nb) {
            int rows[ETA];
            const bool ok = decode_rows<ETA>(E.bits[2 * b], E.bits[2 * b + 1], B.mask0, B.mask1, rows);
            const bool pack = Y >= 4;  // as in k_exact_lu_f32
            uint64_t codes = 0;
            for (int t = 0; t < Y; ++t) {
                const size_t z = (size_t)chunk * Y + t;
                float2 det = make_float2(0.f, 0.f);
                uint16_t ec = 0;
                if (ok) {
                    const float2* Mt = smQ + (size_t)t * n * S;
                    float2 A[ETA][ETA];
#pragma unroll
                    for (int i = 0; i < ETA; ++i) {
                        const float2* rp = Mt + rows[i] * S;
#pragma unroll
                        for (int j = 0; j < ETA; ++j) A[i][j] = rp[j];
                    }
                    float er2, zabs2;
                    det = lu_det_regs<float, ETA>(A, er2, zabs2);
                    ec = err_term_code(det, er2, zabs2);
                }
                const size_t o = dix(b, (uint32_t)z, B.r);
                B.D32[o] = det;
                if (!pack) {
                    B.E32[o] = ec;
                } else {
                    codes = (codes >> 16) | ((uint64_t)ec << 48);
                    if ((t & 3) == 3) *reinterpret_cast<uint64_t*>(B.E32 + o - 3) = codes;
                }
            }
        }
        __syncthreads();
    }
}

template <int ETA>
static cudaError_t launch_queue_eta(const QueueEntry* q, int nq, int64_t n_items, unsigned long long* head,
                                    size_t smem, int grid, cudaStream_t s) {
    cudaError_t e = raise_dynamic_smem((const void*)k_queue_lu_f32<ETA>, smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {  // one wave of resident CTAs
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_queue_lu_f32<ETA>, 128, smem)) != cudaSuccess)
            return e;
        grid = sms * std::max(1, occ);
    }
    k_queue_lu_f32<ETA><<<grid, 128, smem, s>>>(q, nq, n_items, head);
    return cudaGetLastError();
}

cudaError_t launch_queue_lu_f32(int eta, const QueueEntry* q, int nq, int64_t n_items, unsigned long long* head,
                                size_t smem, int grid, cudaStream_t s, LaunchStats& st) {
    if (n_items <= 0 || nq <= 0) return cudaSuccess;
    cudaError_t e;
    switch (eta) {
        case 1: e = launch_queue_eta<1>(q, nq, n_items, head, smem, grid, s); break;
        case 2: e = launch_queue_eta<2>(q, nq, n_items, head, smem, grid, s); break;
        case 3: e = launch_queue_eta<3>(q, nq, n_items, head, smem, grid, s); break;
        case 4: e = launch_queue_eta<4>(q, nq, n_items, head, smem, grid, s); break;
        case 5: e = launch_queue_eta<5>(q, nq, n_items, head, smem, grid, s); break;
        case 6: e = launch_queue_eta<6>(q, nq, n_items, head, smem, grid, s); break;
        case 7: e = launch_queue_eta<7>(q, nq, n_items, head, smem, grid, s); break;
        case 8: e = launch_queue_eta<8>(q, nq, n_items, head, smem, grid, s); break;
        case 9: e = launch_queue_eta<9>(q, nq, n_items, head, smem, grid, s); break;
        case 10: e = launch_queue_eta<10>(q, nq, n_items, head, smem, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    st.launches += 1;
    return e;
}

}  // namespace ef
