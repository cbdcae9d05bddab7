// Raw Estimate (Section III-A/B, Eqs. 10-12) on the GPU.
//
// One CTA handles one bitstring b and a chunk of its trajectories; every
// thread draws whole trajectories (Philox4x32-10 words against integer
// thresholds, one word per controlled-phase gate) and evaluates
// Y_s = w(x_s)/P_T(x_s) prod_B det U_B(x_s)[R_B, C_B].
//
// Trajectory minors are low-rank corrections of the no-flip minor. Writing
// the block's branch matrix as U(x) = T_L W_L T_{L-1} ... T_1 W_1 T_0 with
// W_l = I - 2 E_{N_l} (N_l = modes whose sign flips in layer l, Section IV-B,
// Eqs. 15-18) and Pi_{a..b} = T_a ... T_b, the minor is
//   A(x) = A0 + sum_l H_l Pi_{l-1..0}[N_l, C],
//   H_l  = -2 (Pi_{L..l}[R, N_l] + sum_{l' > l} H_{l'} Pi_{l'-1..l}[N_{l'}, N_l]),
// with A0 = Pi_{L..0}[R, C]. Each flipped mode costs one rank-one update, so
// a trajectory with few flips needs a handful of eta^2 updates and one LU.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ef_common.cuh"
#include "ef_internal.h"

namespace ef {

__host__ __device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

template <typename R, int ETA>
__global__ void __launch_bounds__(128) k_approx(ApproxDev A, const uint64_t* __restrict__ bits, int64_t nb) {
    using T = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ double red[5][128];
    __shared__ unsigned long long cnt_red[2];

    const int64_t b = blockIdx.x;
    const int chunk = blockIdx.y;
    const int tid = threadIdx.x;
    const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
    double* outp = A.part + ((size_t)b * A.n_chunks + chunk) * 8;

    bool ok = ((w0 & A.inactive0) == 0) && ((w1 & A.inactive1) == 0);
    for (int B = 0; B < A.nblocks; ++B)
        ok = ok && (__popcll(w0 & A.blk[B].mask0) + __popcll(w1 & A.blk[B].mask1) == A.blk[B].eta);
    if (!ok) {
        if (tid < 8) outp[tid] = 0.0;
        return;
    }

    // shared layout: thresholds (padded to 4), then per block A0[ETA][ETA] and
    // LeftRows[L][ETA][n] = Pi_{L..l}[R, :] for l = 1..L
    const int k = A.k;
    const int k4 = (k + 3) & ~3;
    uint32_t* sT = reinterpret_cast<uint32_t*>(sm_raw);
    T* sA0[kMaxBlocks];
    T* sLeft[kMaxBlocks];
    {
        size_t off = ((size_t)k4 * sizeof(uint32_t) + 15) & ~(size_t)15;
        for (int B = 0; B < kMaxBlocks; ++B) {
            sA0[B] = reinterpret_cast<T*>(sm_raw + off);
            if (B < A.nblocks) off += (size_t)ETA * ETA * sizeof(T) + (size_t)A.blk[B].L * ETA * A.blk[B].n * sizeof(T);
            sLeft[B] = sA0[B] + ETA * ETA;
        }
    }
    for (int j = tid; j < k4; j += blockDim.x) sT[j] = (j < k) ? A.T[j] : 0u;

    for (int B = 0; B < A.nblocks; ++B) {
        const ApproxBlockDev& blk = A.blk[B];
        int cnt;
        const T* P = reinterpret_cast<const T*>(blk.P);
        const int n = blk.n, L = blk.L;
        const T* PL0 = P + (size_t)tri(L, 0) * n * n;
        for (int e = tid; e < ETA * ETA; e += blockDim.x) {
            const int i = e / ETA, j = e - i * ETA;
            T v = mk(R(i == j ? 1 : 0), R(0));
            if (i < blk.eta && j < blk.eta) {
                const int ri = nth_row(w0, w1, blk.mask0, blk.mask1, i, cnt);
                v = PL0[(size_t)ri * n + blk.cols[j]];
            } else if (i < blk.eta || j < blk.eta) {
                v = mk(R(0), R(0));
            }
            sA0[B][e] = v;
        }
        for (int e = tid; e < L * ETA * n; e += blockDim.x) {
            const int l = e / (ETA * n);
            const int rem = e - l * ETA * n;
            const int i = rem / n, m = rem - i * n;
            T v = mk(R(0), R(0));
            if (i < blk.eta) {
                const int ri = nth_row(w0, w1, blk.mask0, blk.mask1, i, cnt);
                v = P[(size_t)tri(L, l + 1) * n * n + (size_t)ri * n + m];
            }
            sLeft[B][e] = v;
        }
    }
    __syncthreads();

    // no-flip determinants (every thread computes the same values)
    T det0[kMaxBlocks];
    double y0r = A.R0, y0i = 0.0;
    for (int B = 0; B < A.nblocks; ++B) {
        T M[ETA][ETA];
#pragma unroll
        for (int i = 0; i < ETA; ++i)
#pragma unroll
            for (int j = 0; j < ETA; ++j) M[i][j] = sA0[B][i * ETA + j];
        R er2, zabs2;
        det0[B] = lu_det_regs<R, ETA>(M, er2, zabs2);
        const double dr = (double)det0[B].x, di = (double)det0[B].y;
        const double nr = y0r * dr - y0i * di;
        y0i = y0r * di + y0i * dr;
        y0r = nr;
    }

    const uint32_t blo = (uint32_t)(A.index_base + (uint64_t)b);
    const uint32_t bhi = (uint32_t)((A.index_base + (uint64_t)b) >> 32);
    const int64_t s_begin = (int64_t)chunk * A.traj_per_cta;
    const int64_t s_end = min(A.t, s_begin + (int64_t)A.traj_per_cta);
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    unsigned long long nflips_tot = 0, nlu = 0;
    uint64_t N[kMaxBlocks][kMaxApproxLayers];
    T hs[kMaxApproxStored][ETA];
    int htag[kMaxApproxStored];

    for (int64_t s = s_begin + tid; s < s_end; s += blockDim.x) {
        // ---- sample the trajectory (Eq. 12 with integer thresholds)
        int nflip = 0;
        double rq = 1.0;
        uint32_t lflag[kMaxBlocks] = {};
        for (int q4 = 0; q4 < k4 / 4; ++q4) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)q4, (uint32_t)s, blo, bhi), A.key0, A.key1);
            const int j0 = 4 * q4;
            uint32_t hit = (uint32_t)(u.x < sT[j0]) | ((uint32_t)(u.y < sT[j0 + 1]) << 1) |
                           ((uint32_t)(u.z < sT[j0 + 2]) << 2) | ((uint32_t)(u.w < sT[j0 + 3]) << 3);
            while (hit) {
                const int w = __ffs(hit) - 1;
                hit &= hit - 1;
                const int j = j0 + w;
                ++nflip;
                rq *= A.qratio[j];
                for (int B = 0; B < A.nblocks; ++B) {
                    const int l = A.glayer[B * k + j];
                    if (l) {
                        const uint32_t bit = 1u << (l - 1);
                        if (!(lflag[B] & bit)) N[B][l - 1] = 0;
                        lflag[B] |= bit;
                        N[B][l - 1] ^= A.gmodes[B * k + j];
                    }
                }
            }
        }
        nflips_tot += nflip;

        // ---- block minors
        double dr = 1.0, di = 0.0;
        for (int B = 0; B < A.nblocks; ++B) {
            T det;
            if (lflag[B] == 0) {
                det = det0[B];
            } else {
                const ApproxBlockDev& blk = A.blk[B];
                const int n = blk.n, L = blk.L, eb = blk.eta;
                const T* P = reinterpret_cast<const T*>(blk.P);
                const T* RC = reinterpret_cast<const T*>(blk.RC);
                T M[ETA][ETA];
#pragma unroll
                for (int i = 0; i < ETA; ++i)
#pragma unroll
                    for (int j = 0; j < ETA; ++j) M[i][j] = sA0[B][i * ETA + j];
                int nst = 0;
                for (int l = L; l >= 1; --l) {
                    if (!((lflag[B] >> (l - 1)) & 1u)) continue;
                    uint64_t Nl = N[B][l - 1];
                    const bool store = (lflag[B] & ((1u << (l - 1)) - 1u)) != 0;
                    const int nabove = nst;  // columns of the layers above l only
                    while (Nl) {
                        const int i = __ffsll((long long)Nl) - 1;
                        Nl &= Nl - 1;
                        T h[ETA];
                        const T* left = sLeft[B] + (size_t)(l - 1) * ETA * n;
#pragma unroll
                        for (int r = 0; r < ETA; ++r) h[r] = left[r * n + i];
                        for (int st = 0; st < nabove; ++st) {
                            const int ls = htag[st] >> 8, is = htag[st] & 255;
                            const T mid = P[(size_t)tri(ls - 1, l) * n * n + (size_t)is * n + i];
#pragma unroll
                            for (int r = 0; r < ETA; ++r) h[r] = cfma(h[r], hs[st][r], mid);
                        }
#pragma unroll
                        for (int r = 0; r < ETA; ++r) h[r] = mk(R(-2) * h[r].x, R(-2) * h[r].y);
                        const T* rc = RC + ((size_t)(l - 1) * n + i) * eb;
#pragma unroll
                        for (int c = 0; c < ETA; ++c) {
                            if (c < eb) {
                                const T v = rc[c];
#pragma unroll
                                for (int r = 0; r < ETA; ++r) M[r][c] = cfma(M[r][c], h[r], v);
                            }
                        }
                        if (store && nst < kMaxApproxStored) {
#pragma unroll
                            for (int r = 0; r < ETA; ++r) hs[nst][r] = h[r];
                            htag[nst] = (l << 8) | i;
                            ++nst;
                        }
                    }
                }
                R er2, zabs2;
                det = lu_det_regs<R, ETA>(M, er2, zabs2);
                ++nlu;
            }
            const double xr = (double)det.x, xi = (double)det.y;
            const double t2 = dr * xr - di * xi;
            di = dr * xi + di * xr;
            dr = t2;
        }
        const double mag = A.R0 * rq;
        const double2 Y = times_i_pow(make_double2(mag * dr, mag * di), nflip);
        const double Dr = Y.x - y0r, Di = Y.y - y0i;
        acc[0] += Dr;
        acc[1] += Di;
        acc[2] = fma(Dr, Dr, acc[2]);
        acc[3] = fma(Di, Di, acc[3]);
        acc[4] = fma(Dr, Di, acc[4]);
    }

    // ---- deterministic CTA reduction
    for (int e = 0; e < 5; ++e) red[e][tid] = acc[e];
    if (tid == 0) cnt_red[0] = cnt_red[1] = 0ull;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (tid < off)
            for (int e = 0; e < 5; ++e) red[e][tid] += red[e][tid + off];
        __syncthreads();
    }
    atomicAdd(&cnt_red[0], nflips_tot);
    atomicAdd(&cnt_red[1], nlu);
    __syncthreads();
    if (tid == 0) {
        for (int e = 0; e < 5; ++e) outp[e] = red[e][0];
        outp[5] = y0r;
        outp[6] = y0i;
        outp[7] = 1.0;
        atomicAdd(&A.counters[0], cnt_red[0]);
        atomicAdd(&A.counters[1], cnt_red[1] + (chunk == 0 ? (unsigned long long)A.nblocks : 0ull));
    }
}

template <typename R, int ETA>
static cudaError_t launch_approx_eta(const ApproxDev& a, const uint64_t* bits, int64_t nb, cudaStream_t s) {
    size_t smem = ((size_t)((a.k + 3) & ~3) * sizeof(uint32_t) + 15) & ~(size_t)15;
    for (int B = 0; B < a.nblocks; ++B)
        smem += (size_t)ETA * ETA * sizeof(cplx_t<R>) + (size_t)a.blk[B].L * ETA * a.blk[B].n * sizeof(cplx_t<R>);
    cudaError_t e = raise_dynamic_smem((const void*)k_approx<R, ETA>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)nb, (unsigned)a.n_chunks);
    k_approx<R, ETA><<<grid, 128, smem, s>>>(a, bits, nb);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_approx_r(const ApproxDev& a, const uint64_t* bits, int64_t nb, int eta, cudaStream_t s) {
    switch (eta) {
        case 1: return launch_approx_eta<R, 1>(a, bits, nb, s);
        case 2: return launch_approx_eta<R, 2>(a, bits, nb, s);
        case 3: return launch_approx_eta<R, 3>(a, bits, nb, s);
        case 4: return launch_approx_eta<R, 4>(a, bits, nb, s);
        case 5: return launch_approx_eta<R, 5>(a, bits, nb, s);
        case 6: return launch_approx_eta<R, 6>(a, bits, nb, s);
        case 7: return launch_approx_eta<R, 7>(a, bits, nb, s);
        case 8: return launch_approx_eta<R, 8>(a, bits, nb, s);
        default: return cudaErrorInvalidValue;
    }
}

// FP32 minors up to 13 particles per block (the matrix partly lives in local memory)
template <>
cudaError_t launch_approx_r<float>(const ApproxDev& a, const uint64_t* bits, int64_t nb, int eta, cudaStream_t s) {
    switch (eta) {
        case 1: return launch_approx_eta<float, 1>(a, bits, nb, s);
        case 2: return launch_approx_eta<float, 2>(a, bits, nb, s);
        case 3: return launch_approx_eta<float, 3>(a, bits, nb, s);
        case 4: return launch_approx_eta<float, 4>(a, bits, nb, s);
        case 5: return launch_approx_eta<float, 5>(a, bits, nb, s);
        case 6: return launch_approx_eta<float, 6>(a, bits, nb, s);
        case 7: return launch_approx_eta<float, 7>(a, bits, nb, s);
        case 8: return launch_approx_eta<float, 8>(a, bits, nb, s);
        case 9: return launch_approx_eta<float, 9>(a, bits, nb, s);
        case 10: return launch_approx_eta<float, 10>(a, bits, nb, s);
        case 11: return launch_approx_eta<float, 11>(a, bits, nb, s);
        case 12: return launch_approx_eta<float, 12>(a, bits, nb, s);
        case 13: return launch_approx_eta<float, 13>(a, bits, nb, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_approx(const ApproxDev& a, const uint64_t* bits, int64_t nb, bool fp64, cudaStream_t s,
                          LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    int eta = 1;
    for (int B = 0; B < a.nblocks; ++B) eta = std::max(eta, a.blk[B].eta);
    if (eta > (fp64 ? kMaxApproxEta64 : kMaxApproxEta)) return cudaErrorInvalidValue;
    cudaError_t e = fp64 ? launch_approx_r<double>(a, bits, nb, eta, s) : launch_approx_r<float>(a, bits, nb, eta, s);
    st.launches += 1;
    return e;
}

// alpha_hat = Y0 + sum D / t; p_hat = |alpha_hat|^2;
// stderr = 2 sqrt(Var[Re(conj(alpha_hat) Y)] / t) from the shifted sums.
__global__ void k_approx_finalize(ApproxDev A, int64_t nb, double* __restrict__ out, double* __restrict__ se) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double* p = A.part + (size_t)b * A.n_chunks * 8;
    if (p[7] == 0.0) {
        out[b] = 0.0;
        if (se) se[b] = 0.0;
        return;
    }
    double s[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < A.n_chunks; ++c)
        for (int e = 0; e < 5; ++e) s[e] += p[(size_t)c * 8 + e];
    const double t = (double)A.t;
    const double ar = p[5] + s[0] / t, ai = p[6] + s[1] / t;
    out[b] = ar * ar + ai * ai;
    if (se) {
        double v = 0.0;
        if (A.t > 1) {
            const double vr = (s[2] - s[0] * s[0] / t) / (t - 1.0);
            const double vi = (s[3] - s[1] * s[1] / t) / (t - 1.0);
            const double cv = (s[4] - s[0] * s[1] / t) / (t - 1.0);
            v = ar * ar * vr + ai * ai * vi + 2.0 * ar * ai * cv;
        }
        se[b] = 2.0 * sqrt(fmax(v, 0.0) / t);
    }
}

cudaError_t launch_approx_finalize(const ApproxDev& a, int64_t nb, double* out, double* stderr_out, cudaStream_t s,
                                   LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    k_approx_finalize<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(a, nb, out, stderr_out);
    st.launches += 1;
    return cudaGetLastError();
}

}  // namespace ef
