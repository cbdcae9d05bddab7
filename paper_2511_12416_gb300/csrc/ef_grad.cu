// Adjoint of the Exact probabilities (vector-Jacobian product, FP64).
//
// With L = sum_b g_b p_b and p_b = |amp_b|^2, dL = Re sum_b gamma_b d amp_b,
// gamma_b = 2 g_b conj(amp_b). The forward structure (see ef_exact.cu) is
//   amp = sum_{x_sh} w_sh(x_sh) prod_B A_B(x_sh),
//   A_B(x_sh) = sum_{z local} Omega_B(z) det_B(z ^ s_B(x_sh)),
//   det_B(z) = det U_B(z)[R, C],  U_B(z)[:, C] = T_L W_L(z) ... T_1 W_1(z) S_0[:, C].
// The kernels here produce, deterministically (fixed summation orders, no
// floating-point atomics):
//   * k_grad_combine : per bitstring, amp, p, gamma and the cotangent of every
//     minor, gamma C_B(z) with C_B(z) = d amp / d det_B(z); the cotangents of
//     the weight tables, gamma E_B(z_local) and gamma A_0 A_1 (x_sh);
//   * k_grad_minors  : per (block, pattern), Ubar(z) = sum_b cot_b(z) adj(A_b)^T
//     scattered to the bitstring's rows (d det = sum adj(A)_ji dA_ij), then
//     the reverse sweep through the layers by recomputation, giving each
//     pattern's contribution to Tbar_l and to Sbar_0[:, C];
//   * k_sum_rows     : fixed-order sums of those contributions.
// The host finishes the chain rule through T_l = S_l diag(phases), the
// products of gate matrices in each segment and the weight tables.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ef_common.cuh"
#include "ef_internal.h"

namespace ef {

__device__ __forceinline__ double2 cm2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int NT>
__device__ __forceinline__ double block_sum_g(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int off = NT / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- combine with cotangents
__global__ void __launch_bounds__(256) k_grad_combine(GradDev G, const uint64_t* __restrict__ bits, int64_t nb,
                                                      const double* __restrict__ grad_p, double* __restrict__ out_p) {
    constexpr int NT = 256;
    extern __shared__ double2 smA[];  // A_0[2^k_sh], A_1[2^k_sh]
    __shared__ double red[NT];
    __shared__ double2 s_gamma;
    const ExactCombineDev& C = G.cm;
    const int tid = threadIdx.x;
    const int nsh = 1 << C.k_sh;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
        bool ok = ((w0 & C.inactive0) == 0) && ((w1 & C.inactive1) == 0);
        for (int B = 0; B < C.nblocks; ++B)
            ok = ok && (__popcll(w0 & C.mask[B][0]) + __popcll(w1 & C.mask[B][1]) == C.eta[B]);
        double ar = 0.0, ai = 0.0;
        if (ok) {
            if (C.nblocks == 0) {
                ar = tid == 0 ? 1.0 : 0.0;
            } else if (C.nblocks == 1) {
                for (int z = tid; z < (1 << C.r[0]); z += NT) {
                    const double2 v = C.D64[0][dix(b, (uint32_t)z, C.r[0])];
                    const double2 w = C.Omega[0][z];
                    ar = fma(w.x, v.x, fma(-w.y, v.y, ar));
                    ai = fma(w.x, v.y, fma(w.y, v.x, ai));
                }
            } else {
                for (int xs = tid; xs < nsh; xs += NT) {
                    double2 a[2];
                    for (int B = 0; B < 2; ++B) {
                        const uint32_t sB = C.s[B][xs];
                        double sx = 0.0, sy = 0.0;
                        for (int zl = 0; zl < (1 << C.r_loc[B]); ++zl) {
                            const double2 v = C.D64[B][dix(b, (uint32_t)zl ^ sB, C.r[B])];
                            const double2 w = C.Omega[B][zl];
                            sx = fma(w.x, v.x, fma(-w.y, v.y, sx));
                            sy = fma(w.x, v.y, fma(w.y, v.x, sy));
                        }
                        a[B] = make_double2(sx, sy);
                        smA[B * nsh + xs] = a[B];
                    }
                    const double2 t = cm2(C.WS[xs], cm2(a[0], a[1]));
                    ar += t.x;
                    ai += t.y;
                }
            }
        }
        ar = block_sum_g<NT>(ar, red);
        ai = block_sum_g<NT>(ai, red);
        if (tid == 0) {
            const double p = ok ? ar * ar + ai * ai : 0.0;
            if (out_p) out_p[b] = p;
            const double g2 = ok ? 2.0 * grad_p[b] : 0.0;
            s_gamma = make_double2(g2 * ar, -g2 * ai);  // 2 g conj(amp)
        }
        __syncthreads();
        const double2 gam = s_gamma;
        // minor cotangents gamma C_B(z) and local-weight cotangents gamma E_B(zl)
        for (int B = 0; B < C.nblocks; ++B) {
            const int nz = 1 << C.r[B];
            const uint32_t lmask = (1u << C.r_loc[B]) - 1u;
            const double2* Aoth = smA + (1 - B) * nsh;
            for (int z = tid; z < nz; z += NT) {
                double2 cz = make_double2(0.0, 0.0);
                if (ok) {
                    if (C.nblocks == 1) {
                        cz = C.Omega[0][z];
                    } else {
                        const uint32_t h = (uint32_t)z >> C.r_loc[B];
                        for (uint32_t g = C.goff[B][h]; g < C.goff[B][h + 1]; ++g) {
                            const uint32_t xs = C.perm[B][g];
                            const uint32_t zl = ((uint32_t)z ^ C.s[B][xs]) & lmask;
                            const double2 t = cm2(C.WS[xs], cm2(C.Omega[B][zl], Aoth[xs]));
                            cz.x += t.x;
                            cz.y += t.y;
                        }
                    }
                }
                G.cot[B][(size_t)z * nb + b] = cm2(gam, cz);
            }
            if (C.nblocks == 1) {
                const int nzl = 1 << C.r_loc[0];
                for (int zl = tid; zl < nzl; zl += NT) {
                    const double2 v = ok ? C.D64[0][dix(b, (uint32_t)zl, C.r[0])] : make_double2(0.0, 0.0);
                    G.ebar[0][(size_t)b * nzl + zl] = cm2(gam, v);
                }
            }
        }
        if (C.nblocks == 2) {
            // E_B(zl) = sum_xs w_sh(xs) A_other(xs) det_B(zl ^ s_B(xs)): one warp per
            // (block, zl), lanes over xs, then a butterfly (full warps: on this GPU an
            // FP64 instruction costs the same with one active lane as with 32)
            const int lane = tid & 31, warp = tid >> 5;
            const int nz0 = 1 << C.r_loc[0], nz1 = 1 << C.r_loc[1];
            for (int pr = warp; pr < nz0 + nz1; pr += NT / 32) {
                const int B = pr < nz0 ? 0 : 1;
                const int zl = B ? pr - nz0 : pr;
                const double2* Aoth = smA + (1 - B) * nsh;
                double ex = 0.0, ey = 0.0;
                if (ok)
                    for (int xs = lane; xs < nsh; xs += 32) {
                        const double2 v = C.D64[B][dix(b, (uint32_t)zl ^ C.s[B][xs], C.r[B])];
                        const double2 t = cm2(C.WS[xs], cm2(Aoth[xs], v));
                        ex += t.x;
                        ey += t.y;
                    }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    ex += __shfl_xor_sync(0xffffffffu, ex, off);
                    ey += __shfl_xor_sync(0xffffffffu, ey, off);
                }
                if (lane == 0) G.ebar[B][(size_t)b * (B ? nz1 : nz0) + zl] = cm2(gam, make_double2(ex, ey));
            }
        }
        if (C.nblocks == 2)
            for (int xs = tid; xs < nsh; xs += NT)
                G.pbar[(size_t)b * nsh + xs] = ok ? cm2(gam, cm2(smA[xs], smA[nsh + xs])) : make_double2(0.0, 0.0);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- minor adjoints per pattern

// In-place Gauss-Jordan inversion with partial (row) pivoting: A becomes
// A^{-1}, the return value is det(A) (0 for an exactly singular pivot column,
// A then undefined). Each step scales the pivot row and clears column k in all
// other rows, N^3 complex multiply-adds in all (half of the work of reducing
// [A | I]); the row interchanges are undone on the inverse's columns in
// reverse order.
template <int N>
__device__ __forceinline__ double2 inv_det_inplace(double2 (&A)[N][N]) {
    double2 det = make_double2(1.0, 0.0);
    bool odd = false;
    int perm[N];
    for (int k = 0; k < N; ++k) {
        double best = abs2(A[k][k]);
        int p = k;
        for (int i = k + 1; i < N; ++i) {
            const double m = abs2(A[i][k]);
            if (m > best) {
                best = m;
                p = i;
            }
        }
        if (best == 0.0) return make_double2(0.0, 0.0);
        perm[k] = p;
        if (p != k) {
            odd = !odd;
            for (int j = 0; j < N; ++j) {
                const double2 t = A[k][j];
                A[k][j] = A[p][j];
                A[p][j] = t;
            }
        }
        const double2 piv = A[k][k];
        det = cm2(det, piv);
        const double ib = 1.0 / best;
        const double2 ip = make_double2(piv.x * ib, -piv.y * ib);
        A[k][k] = make_double2(1.0, 0.0);
        for (int j = 0; j < N; ++j) A[k][j] = cm2(A[k][j], ip);
        for (int i = 0; i < N; ++i) {
            if (i == k) continue;
            const double2 f = A[i][k];
            A[i][k] = make_double2(0.0, 0.0);
            for (int j = 0; j < N; ++j) A[i][j] = cfms(A[i][j], f, A[k][j]);
        }
    }
    for (int k = N - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p == k) continue;
        for (int i = 0; i < N; ++i) {
            const double2 t = A[i][k];
            A[i][k] = A[i][p];
            A[i][p] = t;
        }
    }
    return odd ? make_double2(-det.x, -det.y) : det;
}

template <int N>
__device__ double2 cofactor(const double2* __restrict__ Mz, const int (&rows)[N], int i0, int j0) {
    constexpr int K = N - 1;
    if constexpr (K == 0) {
        return make_double2(1.0, 0.0);
    } else {
        double2 S[K][K];
        for (int i = 0, ii = 0; i < N; ++i) {
            if (i == i0) continue;
            for (int j = 0, jj = 0; j < N; ++j) {
                if (j == j0) continue;
                S[ii][jj++] = Mz[rows[i] * N + j];
            }
            ++ii;
        }
        double2 det = make_double2(((i0 + j0) & 1) ? -1.0 : 1.0, 0.0);
        for (int k = 0; k < K; ++k) {
            int p = k;
            double best = abs2(S[k][k]);
            for (int i = k + 1; i < K; ++i)
                if (abs2(S[i][k]) > best) {
                    best = abs2(S[i][k]);
                    p = i;
                }
            if (best == 0.0) return make_double2(0.0, 0.0);
            if (p != k) {
                det = make_double2(-det.x, -det.y);
                for (int j = 0; j < K; ++j) {
                    const double2 t = S[k][j];
                    S[k][j] = S[p][j];
                    S[p][j] = t;
                }
            }
            det = cm2(det, S[k][k]);
            const double ib = 1.0 / best;
            const double2 ip = make_double2(S[k][k].x * ib, -S[k][k].y * ib);
            for (int i = k + 1; i < K; ++i) {
                const double2 l = cm2(S[i][k], ip);
                for (int j = k + 1; j < K; ++j) S[i][j] = cfms(S[i][j], l, S[k][j]);
            }
        }
        return det;
    }
}

// The cofactor path for a singular minor, kept out of line: inlined next to
// the in-place inverse it made k_grad_minors<6> spill 4.4 KB per thread. The
// rows are passed as the bitstring's local row mask (ascending set bits), so
// that no register array of the caller has its address taken.
template <int N>
__device__ __noinline__ double2 cofactor_of_mask(const double2* __restrict__ Mz, uint64_t lm, int i0, int j0) {
    int rows[N];
    for (int i = 0; i < N; ++i) {
        rows[i] = __ffsll((long long)lm) - 1;
        lm &= lm - 1;
    }
    return cofactor<N>(Mz, rows, i0, j0);
}

template <int ETA>
__global__ void __launch_bounds__(128) k_grad_minors(GradDev G, int blk, const uint64_t* __restrict__ bits,
                                                     int64_t nb) {
    constexpr int NT = 128;
    const ExactBlockDev& B = G.blk[blk];
    const int n = B.n, L = B.L;
    const int ne = n * ETA;
    extern __shared__ double2 sm[];
    // per-thread cotangent blocks, GS (odd) double2 apart so that a warp's
    // stores of one (i, j) spread over every bank (ETA^2 apart: up to 16-way)
    constexpr int GS = (ETA * ETA) | 1;
    double2* gs = sm;                                  // [NT][GS]
    double2* ubar = gs + NT * GS;                      // [n][ETA]
    double2* xs = ubar + ne;                           // [L+1][n][ETA] forward values X_l
    double2* xb = xs + (size_t)(L + 1) * ne;           // [n][ETA] running Xbar
    uint64_t* rmask = reinterpret_cast<uint64_t*>(xb + ne);  // [NT] local row masks
    int* sgn = reinterpret_cast<int*>(rmask + NT);     // [n]
    const int tid = threadIdx.x;
    const uint32_t z = blockIdx.x;
    const double2* Mz = B.M64 + (size_t)z * ne;
    const double2* cot = G.cot[blk] + (size_t)z * nb;
    for (int e = tid; e < ne; e += NT) ubar[e] = make_double2(0.0, 0.0);
    for (int64_t t0 = 0; t0 < nb; t0 += NT) {
        const int64_t b = t0 + tid;
        int rows[ETA];
        uint64_t lm = 0;
        bool ok = false;
        double2* gt = gs + (size_t)tid * GS;
        if (b < nb) {
            ok = decode_rows<ETA>(bits[2 * b], bits[2 * b + 1], B.mask0, B.mask1, rows);
            const double2 cb = cot[b];
            ok = ok && (cb.x != 0.0 || cb.y != 0.0);
            if (ok) {
                double2 A[ETA][ETA];
                for (int i = 0; i < ETA; ++i) {
                    lm |= 1ull << rows[i];
                    for (int j = 0; j < ETA; ++j) A[i][j] = Mz[rows[i] * ETA + j];
                }
                const double2 det = inv_det_inplace<ETA>(A);
                if (det.x != 0.0 || det.y != 0.0) {
                    // G[i][j] = cot det (A^{-1})[j][i] = cot adj(A)_{ji} = cot d det / dA_ij
                    const double2 f = cm2(cb, det);
                    for (int i = 0; i < ETA; ++i)
                        for (int j = 0; j < ETA; ++j) gt[i * ETA + j] = cm2(f, A[j][i]);
                } else {
                    for (int i = 0; i < ETA; ++i)
                        for (int j = 0; j < ETA; ++j) gt[i * ETA + j] = cm2(cb, cofactor_of_mask<ETA>(Mz, lm, i, j));
                }
            }
        }
        rmask[tid] = ok ? lm : 0ull;
        if (!ok)
            for (int e = 0; e < ETA * ETA; ++e) gt[e] = make_double2(0.0, 0.0);
        __syncthreads();
        // fixed-order accumulation: element (m, j) sums the tile's threads in order
        for (int e = tid; e < ne; e += NT) {
            const int m = e / ETA, j = e - m * ETA;
            double2 acc = ubar[e];
            const uint64_t below = (m == 63) ? ~0ull >> 1 : ((1ull << m) - 1ull);
            for (int t = 0; t < NT; ++t) {
                const uint64_t msk = rmask[t];
                if ((msk >> m) & 1ull) {
                    const int i = __popcll(msk & below);
                    const double2 g = gs[(size_t)t * GS + i * ETA + j];
                    acc.x += g.x;
                    acc.y += g.y;
                }
            }
            ubar[e] = acc;
        }
        __syncthreads();
    }
    // forward recomputation X_0 = S_0[:, C], X_l = T_l W_l X_{l-1}
    for (int e = tid; e < ne; e += NT) xs[e] = B.S0C[e];
    __syncthreads();
    for (int l = 0; l < L; ++l) {
        for (int m = tid; m < n; m += NT) sgn[m] = __popc(z & B.F[l * n + m]) & 1;
        __syncthreads();
        const double2* T = B.T + (size_t)l * n * n;
        const double2* cur = xs + (size_t)l * ne;
        double2* nxt = xs + (size_t)(l + 1) * ne;
        for (int e = tid; e < ne; e += NT) {
            const int i = e / ETA, c = e - i * ETA;
            double ax = 0.0, ay = 0.0;
            for (int m = 0; m < n; ++m) {
                const double2 t = T[i * n + m];
                double2 x = cur[m * ETA + c];
                if (sgn[m]) x = make_double2(-x.x, -x.y);
                ax = fma(t.x, x.x, fma(-t.y, x.y, ax));
                ay = fma(t.x, x.y, fma(t.y, x.x, ay));
            }
            nxt[e] = make_double2(ax, ay);
        }
        __syncthreads();
    }
    // reverse sweep: Tbar_l += Xbar_l (W_l X_{l-1})^T, Xbar_{l-1} = W_l T_l^T Xbar_l
    for (int e = tid; e < ne; e += NT) xb[e] = ubar[e];
    __syncthreads();
    for (int l = L - 1; l >= 0; --l) {
        for (int m = tid; m < n; m += NT) sgn[m] = __popc(z & B.F[l * n + m]) & 1;
        __syncthreads();
        const double2* T = B.T + (size_t)l * n * n;
        const double2* prev = xs + (size_t)l * ne;
        double2* tg = G.tbar[blk] + ((size_t)z * L + l) * n * n;
        for (int e = tid; e < n * n; e += NT) {
            const int i = e / n, m = e - i * n;
            double ax = 0.0, ay = 0.0;
            for (int c = 0; c < ETA; ++c) {
                const double2 xbv = xb[i * ETA + c];
                const double2 pv = prev[m * ETA + c];
                ax = fma(xbv.x, pv.x, fma(-xbv.y, pv.y, ax));
                ay = fma(xbv.x, pv.y, fma(xbv.y, pv.x, ay));
            }
            tg[e] = sgn[m] ? make_double2(-ax, -ay) : make_double2(ax, ay);
        }
        __syncthreads();
        // new Xbar into ubar (as scratch), then copy
        for (int e = tid; e < ne; e += NT) {
            const int m = e / ETA, c = e - m * ETA;
            double ax = 0.0, ay = 0.0;
            for (int i = 0; i < n; ++i) {
                const double2 t = T[i * n + m];
                const double2 x = xb[i * ETA + c];
                ax = fma(t.x, x.x, fma(-t.y, x.y, ax));
                ay = fma(t.x, x.y, fma(t.y, x.x, ay));
            }
            ubar[e] = sgn[m] ? make_double2(-ax, -ay) : make_double2(ax, ay);
        }
        __syncthreads();
        for (int e = tid; e < ne; e += NT) xb[e] = ubar[e];
        __syncthreads();
    }
    double2* sg = G.sbar[blk] + (size_t)z * ne;
    for (int e = tid; e < ne; e += NT) sg[e] = xb[e];
}

size_t grad_minors_smem(int n, int eta, int L) {
    const size_t ne = (size_t)n * eta;
    // matches k_grad_minors: [128][(eta^2) | 1] cotangent blocks, ubar, X_0..X_L, Xbar, row masks, signs
    return (size_t)128 * ((eta * eta) | 1) * sizeof(double2) + ne * sizeof(double2) * (3 + L) +
           128 * sizeof(uint64_t) + (size_t)n * sizeof(int);
}

template <int ETA>
static cudaError_t launch_grad_minors_eta(const GradDev& g, int blk, const uint64_t* bits, int64_t nb,
                                          cudaStream_t s) {
    const ExactBlockDev& B = g.blk[blk];
    const size_t smem = grad_minors_smem(B.n, ETA, B.L);
    cudaError_t e = raise_dynamic_smem((const void*)k_grad_minors<ETA>, smem);
    if (e != cudaSuccess) return e;
    k_grad_minors<ETA><<<1u << B.r, 128, smem, s>>>(g, blk, bits, nb);
    return cudaGetLastError();
}

cudaError_t launch_grad(const GradDev& g, const uint64_t* bits, int64_t nb, const double* grad_p, double* out_p,
                        cudaStream_t s, LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    const size_t smem = (size_t)2 * ((size_t)1 << g.cm.k_sh) * sizeof(double2);
    cudaError_t e = raise_dynamic_smem((const void*)k_grad_combine, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)sm_count() * 16));
    k_grad_combine<<<(unsigned)blocks, 256, smem, s>>>(g, bits, nb, grad_p, out_p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    st.launches += 1;
    for (int b = 0; b < g.cm.nblocks; ++b) {
        switch (g.blk[b].eta) {
            case 1: e = launch_grad_minors_eta<1>(g, b, bits, nb, s); break;
            case 2: e = launch_grad_minors_eta<2>(g, b, bits, nb, s); break;
            case 3: e = launch_grad_minors_eta<3>(g, b, bits, nb, s); break;
            case 4: e = launch_grad_minors_eta<4>(g, b, bits, nb, s); break;
            case 5: e = launch_grad_minors_eta<5>(g, b, bits, nb, s); break;
            case 6: e = launch_grad_minors_eta<6>(g, b, bits, nb, s); break;
            case 7: e = launch_grad_minors_eta<7>(g, b, bits, nb, s); break;
            case 8: e = launch_grad_minors_eta<8>(g, b, bits, nb, s); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        st.launches += 1;
        st.executed_lus += nb * ((int64_t)1 << g.blk[b].r);
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- fixed-order sums
// out[e] = sum_{k < count} in[k * stride + e] for e < width (complex), k ascending.
// out[e] = sum_k in[k * stride + e] for e < width, in a fixed order: a CTA
// covers 32 consecutive e (one per lane); warp w adds rows w, w + 32, w + 64,
// ... and warp 0 then adds the 32 warps' partial sums in order. Splitting the
// count over 32 warps keeps the chains of dependent FP64 additions short.
__global__ void __launch_bounds__(1024) k_sum_rows(const double2* __restrict__ in, int64_t count, int64_t stride,
                                                   int64_t width, double2* __restrict__ out) {
    __shared__ double2 part[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    double ax = 0.0, ay = 0.0;
    if (e < width)
        for (int64_t k = w; k < count; k += 32) {
            const double2 v = in[k * stride + e];
            ax += v.x;
            ay += v.y;
        }
    part[w][lane] = make_double2(ax, ay);
    __syncthreads();
    if (w == 0 && e < width) {
        double sx = 0.0, sy = 0.0;
        for (int q = 0; q < 32; ++q) {
            sx += part[q][lane].x;
            sy += part[q][lane].y;
        }
        out[e] = make_double2(sx, sy);
    }
}

cudaError_t launch_sum_rows(const double2* in, int64_t count, int64_t stride, int64_t width, double2* out,
                            cudaStream_t s, LaunchStats& st) {
    if (width <= 0) return cudaSuccess;
    const int64_t blocks = (width + 31) / 32;
    if (blocks > 2147483647ll) return cudaErrorInvalidValue;
    k_sum_rows<<<(unsigned)blocks, 1024, 0, s>>>(in, count, stride, width, out);
    st.launches += 1;
    return cudaGetLastError();
}

}  // namespace ef
