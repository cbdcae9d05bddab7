// Exact algorithm (Section III-B, Eqs. 8-9) on the GPU.
//
// The circuit's modes split into at most two independent blocks (modes joined
// by Givens rotations; controlled-phase gates are diagonal and never join
// them). For a trajectory x the mode matrix is block diagonal, so the minor's
// determinant is the product of the blocks' minors, and each block's factor
// depends only on the bits y of the gates touching that block. Per block:
//
//   1. k_build_branches  : U_B(y)[:, C_B] = T_L W_L(y) ... T_1 W_1(y) S_0[:, C_B]
//      for every sub-branch y (Section IV-B, Eq. 14 generalised: T_l is the
//      passive segment times the layer's base phases, W_l(y) = diag(+-1)).
//   2. k_exact_lu_*      : per (bitstring, chunk of sub-branches) the weighted
//      sum of minors det U_B(y)[R_B(b), C_B] (Eq. 3), LU with partial pivoting.
//   3. k_exact_combine   : amp(b) = sum_{y_sh} w_sh(y_sh) prod_B A_B(b, y_sh),
//      p(b) = |amp(b)|^2, plus the FP32 path's per-result error estimate.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ef_common.cuh"
#include "ef_internal.h"

namespace ef {

// ---------------------------------------------------------------- 1. builder

__global__ void __launch_bounds__(128) k_build_branches(ExactBlockDev B, int want32) {
    extern __shared__ double2 smb[];
    const int n = B.n, eta = B.eta, ne = n * eta;
    double2* bufA = smb;
    double2* bufB = smb + ne;
    int* sgn = reinterpret_cast<int*>(smb + 2 * ne);
    const uint32_t ny = 1u << (B.k_loc + B.k_sh);
    for (uint32_t y = blockIdx.x; y < ny; y += gridDim.x) {
        double2* cur = bufA;
        double2* nxt = bufB;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) cur[e] = B.S0C[e];
        for (int l = 0; l < B.L; ++l) {
            for (int m = threadIdx.x; m < n; m += blockDim.x) sgn[m] = __popc(y & B.F[l * n + m]) & 1;
            __syncthreads();
            const double2* T = B.T + (size_t)l * n * n;
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const int i = e / eta, c = e - i * eta;
                double ax = 0.0, ay = 0.0;
                for (int m = 0; m < n; ++m) {
                    const double2 t = T[i * n + m];
                    double2 x = cur[m * eta + c];
                    if (sgn[m]) {
                        x.x = -x.x;
                        x.y = -x.y;
                    }
                    ax = fma(t.x, x.x, fma(-t.y, x.y, ax));
                    ay = fma(t.x, x.y, fma(t.y, x.x, ay));
                }
                nxt[e] = make_double2(ax, ay);
            }
            __syncthreads();
            double2* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        __syncthreads();
        double2* o64 = B.M64 + (size_t)y * ne;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const double2 v = cur[e];
            o64[e] = v;
            if (want32) B.M32[(size_t)y * ne + e] = make_float2((float)v.x, (float)v.y);
        }
        __syncthreads();
    }
}

cudaError_t launch_build_branches(const ExactBlockDev& b, bool want32, cudaStream_t s, LaunchStats& st) {
    const size_t smem = (size_t)2 * b.n * b.eta * sizeof(double2) + (size_t)b.n * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(k_build_branches, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t ny = 1u << (b.k_loc + b.k_sh);
    const int grid = (int)std::min<uint32_t>(ny, 152u * 16u);
    k_build_branches<<<grid, 128, smem, s>>>(b, want32 ? 1 : 0);
    st.launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- 2a. FP32, thread per minor
// Thread <-> bitstring; the CTA stages one chunk of 2^c_log2 branch matrices
// (row stride ETA|1 float2 so that rows of one chunk fall in distinct banks)
// and every thread walks the chunk, factoring its own minor in registers.

template <int ETA>
__global__ void __launch_bounds__(128) k_exact_lu_f32(ExactBlockDev B, const uint64_t* __restrict__ bits,
                                                      int64_t nb) {
    extern __shared__ float2 smM[];
    constexpr int S = ETA | 1;
    const int n = B.n;
    const int Y = 1 << B.c_log2;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int rows[ETA];
    const bool ok = (b < nb) && decode_rows<ETA>(bits[2 * b], bits[2 * b + 1], B.mask0, B.mask1, rows);
    const uint32_t locmask = (1u << B.k_loc) - 1u;
    const uint32_t lomask = (1u << B.lobits) - 1u;
    for (int chunk = blockIdx.y; chunk < B.n_chunks; chunk += gridDim.y) {
        const float2* src = B.M32 + (size_t)chunk * Y * n * ETA;
        __syncthreads();
        for (int e = threadIdx.x; e < Y * n * ETA; e += blockDim.x) {
            const int row = e / ETA, j = e - row * ETA;
            smM[row * S + j] = src[e];
        }
        __syncthreads();
        if (b >= nb) continue;
        d4 res = make_d4(0.0, 0.0, 0.0, 0.0);
        if (ok) {
            double ar = 0.0, ai = 0.0;
            double ssum = 0.0, esum = 0.0;
            for (int t = 0; t < Y; ++t) {
                const float2* Mt = smM + (size_t)t * n * S;
                float2 A[ETA][ETA];
#pragma unroll
                for (int i = 0; i < ETA; ++i) {
                    const float2* rp = Mt + rows[i] * S;
#pragma unroll
                    for (int j = 0; j < ETA; ++j) A[i][j] = rp[j];
                }
                float er2, zabs2;
                const float2 det = lu_det_regs<float, ETA>(A, er2, zabs2);
                const uint32_t y = (uint32_t)chunk * (uint32_t)Y + (uint32_t)t;
                const uint32_t yl = y & locmask;
                const double wr = B.WLlo[yl & lomask] * B.WLhi[yl >> B.lobits];
                const double2 wd = times_i_pow(make_double2(wr * (double)det.x, wr * (double)det.y), __popc(yl));
                ar += wd.x;
                ai += wd.y;
                const double w2 = wr * wr;
                const double d2 = (double)det.x * det.x + (double)det.y * det.y;
                ssum = fma(w2, d2, ssum);
                esum = fma(w2, fma(d2, (double)er2, (double)zabs2), esum);
            }
            res = make_d4(ar, ai, ssum, esum);
        }
        B.part[(size_t)chunk * nb + b] = res;
    }
}

template <int ETA>
static cudaError_t launch_f32_eta(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, cudaStream_t s) {
    constexpr int S = ETA | 1;
    const size_t smem = (size_t)(1 << b.c_log2) * b.n * S * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_exact_lu_f32<ETA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((nb + 127) / 128), (unsigned)std::min(b.n_chunks, 65535));
    k_exact_lu_f32<ETA><<<grid, 128, smem, s>>>(b, bits, nb);
    return cudaGetLastError();
}

cudaError_t launch_exact_lu_f32(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, cudaStream_t s,
                                LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    cudaError_t e;
    switch (b.eta) {
        case 1: e = launch_f32_eta<1>(b, bits, nb, s); break;
        case 2: e = launch_f32_eta<2>(b, bits, nb, s); break;
        case 3: e = launch_f32_eta<3>(b, bits, nb, s); break;
        case 4: e = launch_f32_eta<4>(b, bits, nb, s); break;
        case 5: e = launch_f32_eta<5>(b, bits, nb, s); break;
        case 6: e = launch_f32_eta<6>(b, bits, nb, s); break;
        case 7: e = launch_f32_eta<7>(b, bits, nb, s); break;
        case 8: e = launch_f32_eta<8>(b, bits, nb, s); break;
        case 9: e = launch_f32_eta<9>(b, bits, nb, s); break;
        case 10: e = launch_f32_eta<10>(b, bits, nb, s); break;
        default: return cudaErrorInvalidValue;
    }
    st.launches += 1;
    st.executed_lus += nb * ((int64_t)b.n_chunks << b.c_log2);
    return e;
}

// ---------------------------------------------------------------- 2b. warp-row LU (FP64, or FP32 for large eta)
// A group of G lanes handles one (bitstring, chunk) work item; lane r holds
// row r of each minor. Work items are visited warp-uniformly in a grid-stride
// loop; in list mode the bitstrings are list[0..*list_count) (the results the
// FP32 path flagged) and partials go to [chunk][list position] with stride cap.

template <typename R, int G>
__global__ void __launch_bounds__(256) k_exact_lu_rows(ExactBlockDev B, const uint64_t* __restrict__ bits,
                                                       int64_t nb, const int* __restrict__ list,
                                                       const int* __restrict__ list_count, int64_t cap,
                                                       const cplx_t<R>* __restrict__ M) {
    using T = cplx_t<R>;
    const int lane = threadIdx.x & 31;
    const int r = lane & (G - 1);
    constexpr int GPW = 32 / G;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    const int64_t stride = list ? cap : nb;
    const int64_t total = count * (int64_t)B.n_chunks;
    const int n = B.n, eta = B.eta;
    const int Y = 1 << B.c_log2;
    const uint32_t locmask = (1u << B.k_loc) - 1u;
    const uint32_t lomask = (1u << B.lobits) - 1u;
    for (int64_t wbase = warp_global * GPW; wbase < total; wbase += nwarps * GPW) {
        const int64_t item = wbase + lane / G;
        const bool valid = item < total;
        const int64_t chunk = valid ? item / count : 0;
        const int64_t pos = valid ? item - chunk * count : 0;
        int row_idx = -1, cnt = -1;
        if (valid) {
            const int64_t b = list ? (int64_t)list[pos] : pos;
            row_idx = nth_row(bits[2 * b], bits[2 * b + 1], B.mask0, B.mask1, r, cnt);
        }
        const bool ok = valid && (cnt == eta);
        double ar = 0.0, ai = 0.0, ssum = 0.0, esum = 0.0;
        for (int t = 0; t < Y; ++t) {
            const uint32_t y = (uint32_t)chunk * (uint32_t)Y + (uint32_t)t;
            T rowv[G];
            const T* src = M + ((size_t)y * n + (size_t)(row_idx < 0 ? 0 : row_idx)) * eta;
            const bool live = ok && r < eta;
#pragma unroll
            for (int j = 0; j < G; ++j) rowv[j] = (live && j < eta) ? src[j] : mk(R(0), R(0));
            R er2, zabs2;
            const T det = lu_det_rows<R, G>(rowv, r, eta, er2, zabs2);
            const uint32_t yl = y & locmask;
            const double wr = B.WLlo[yl & lomask] * B.WLhi[yl >> B.lobits];
            const double2 wd = times_i_pow(make_double2(wr * (double)det.x, wr * (double)det.y), __popc(yl));
            ar += wd.x;
            ai += wd.y;
            const double w2 = wr * wr;
            const double d2 = (double)det.x * det.x + (double)det.y * det.y;
            ssum = fma(w2, d2, ssum);
            esum = fma(w2, fma(d2, (double)er2, (double)zabs2), esum);
        }
        if (valid && r == 0)
            B.part[(size_t)chunk * stride + pos] = ok ? make_d4(ar, ai, ssum, esum) : make_d4(0, 0, 0, 0);
    }
}

template <typename R, int G>
static cudaError_t launch_rows_g(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, int64_t cap, const void* M, cudaStream_t s) {
    const int64_t count = list ? cap : nb;
    const int64_t items = count * (int64_t)b.n_chunks;
    const int64_t warps = (items + (32 / G) - 1) / (32 / G);
    int64_t blocks = (warps + 7) / 8;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, 152 * 16));
    k_exact_lu_rows<R, G><<<(unsigned)blocks, 256, 0, s>>>(b, bits, nb, list, list_count, cap,
                                                          reinterpret_cast<const cplx_t<R>*>(M));
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_rows_r(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, int64_t cap, const void* M, cudaStream_t s) {
    if (b.eta <= 2) return launch_rows_g<R, 2>(b, bits, nb, list, list_count, cap, M, s);
    if (b.eta <= 4) return launch_rows_g<R, 4>(b, bits, nb, list, list_count, cap, M, s);
    if (b.eta <= 8) return launch_rows_g<R, 8>(b, bits, nb, list, list_count, cap, M, s);
    if (b.eta <= 16) return launch_rows_g<R, 16>(b, bits, nb, list, list_count, cap, M, s);
    return launch_rows_g<R, 32>(b, bits, nb, list, list_count, cap, M, s);
}

cudaError_t launch_exact_lu_rows(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, int64_t cap, bool fp64, cudaStream_t s, LaunchStats& st) {
    if ((list ? cap : nb) <= 0) return cudaSuccess;
    if (b.eta > kMaxEtaRows) return cudaErrorInvalidValue;
    cudaError_t e = fp64 ? launch_rows_r<double>(b, bits, nb, list, list_count, cap, b.M64, s)
                         : launch_rows_r<float>(b, bits, nb, list, list_count, cap, b.M32, s);
    st.launches += 1;
    if (!list) st.executed_lus += nb * ((int64_t)b.n_chunks << b.c_log2);
    return e;
}

// ---------------------------------------------------------------- 3. combine

__global__ void __launch_bounds__(256) k_exact_combine(ExactCombineDev C, const uint64_t* __restrict__ bits,
                                                       int64_t nb, const int* __restrict__ list,
                                                       const int* __restrict__ list_count, int64_t stride,
                                                       double* __restrict__ out, double* __restrict__ err,
                                                       int* __restrict__ append_list, int* __restrict__ append_count) {
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < count;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = list ? (int64_t)list[pos] : pos;
        const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
        bool ok = ((w0 & C.inactive0) == 0) && ((w1 & C.inactive1) == 0);
        for (int B = 0; B < C.nblocks; ++B)
            ok = ok && (__popcll(w0 & C.mask[B][0]) + __popcll(w1 & C.mask[B][1]) == C.eta[B]);
        double p = 0.0, e = 0.0;
        if (ok) {
            double ar = 0.0, ai = 0.0, S = 0.0, E = 0.0;
            if (C.nblocks == 0) {
                ar = 1.0;
                S = 1.0;
            } else if (C.nblocks == 1) {
                const int nch = 1 << (C.k_loc[0] + C.k_sh - C.c_log2[0]);
                for (int c = 0; c < nch; ++c) {
                    const d4 v = C.part[0][(size_t)c * stride + pos];
                    ar += v.x;
                    ai += v.y;
                    S += v.z;
                    E += v.w;
                }
            } else {
                const int nys = 1 << C.k_sh;
                const int cpy0 = 1 << (C.k_loc[0] - C.c_log2[0]);
                const int cpy1 = 1 << (C.k_loc[1] - C.c_log2[1]);
                const uint32_t lomask = (1u << C.shlobits) - 1u;
                for (int ys = 0; ys < nys; ++ys) {
                    double a0r = 0, a0i = 0, s0 = 0, e0 = 0, a1r = 0, a1i = 0, s1 = 0, e1 = 0;
                    for (int c = ys * cpy0; c < (ys + 1) * cpy0; ++c) {
                        const d4 v = C.part[0][(size_t)c * stride + pos];
                        a0r += v.x; a0i += v.y; s0 += v.z; e0 += v.w;
                    }
                    for (int c = ys * cpy1; c < (ys + 1) * cpy1; ++c) {
                        const d4 v = C.part[1][(size_t)c * stride + pos];
                        a1r += v.x; a1i += v.y; s1 += v.z; e1 += v.w;
                    }
                    const double wr = C.WSlo[ys & lomask] * C.WShi[(uint32_t)ys >> C.shlobits];
                    const double2 prod = times_i_pow(make_double2(a0r * a1r - a0i * a1i, a0r * a1i + a0i * a1r),
                                                     __popc((unsigned)ys));
                    ar = fma(wr, prod.x, ar);
                    ai = fma(wr, prod.y, ai);
                    const double w2 = wr * wr;
                    S = fma(w2, s0 * s1, S);
                    E = fma(w2, e0 * s1 + s0 * e1, E);
                }
            }
            p = ar * ar + ai * ai;
            // rounding errors of different minors are independent: the FP32
            // amplitude error is estimated in quadrature, |d amp| ~ K eta u sqrt(2 E)
            const double dabs = 2.0 * sqrt(p) * C.err_coef * sqrt(2.0 * E);
            e = dabs / fmax(p, C.p_floor);
        }
        out[b] = p;
        if (list) {
            if (err) err[b] = -fabs(err[b]);
        } else {
            if (err) err[b] = e;
            if (append_list && e > C.tol) {
                const int idx = atomicAdd(append_count, 1);
                append_list[idx] = (int)b;
            }
        }
    }
}

cudaError_t launch_exact_combine(const ExactCombineDev& c, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, double* out, double* err, int* append_list,
                                 int* append_count, cudaStream_t s, LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    int64_t blocks = (nb + 255) / 256;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, 152 * 32));
    // in list mode the partial stride is the list capacity (= nb)
    k_exact_combine<<<(unsigned)blocks, 256, 0, s>>>(c, bits, nb, list, list_count, nb, out, err, append_list,
                                                     append_count);
    st.launches += 1;
    return cudaGetLastError();
}

}  // namespace ef
