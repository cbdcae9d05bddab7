// Raw Estimate (Section III-A/B, Eqs. 10-12) on the GPU.
//
// Work items are (bitstring b, chunk of its trajectories); a CTA takes items
// in turn. Every thread draws whole trajectories (Philox4x32-10 words against
// integer thresholds, one word per controlled-phase gate) and evaluates
// Y_s = w(x_s)/P_T(x_s) prod_B det U_B(x_s)[R_B, C_B].
//
// Trajectory minors against the no-flip minor. Per mode block the branch
// matrix is U(x) = T_L W_L T_{L-1} ... T_1 W_1 T_0 with W_l = I - 2 E_{N_l}
// (N_l = modes whose sign flips in layer l, Section IV-B, Eqs. 15-18) and
// Pi_{a..b} = T_a ... T_b. With A0 = Pi_{L..0}[R, C], Lambda_l = Pi_{L..l}[R, :]
// and rho_l = Pi_{l-1..0}[:, C], the minor is a low-rank change of A0,
//   A(x) = A0 + H Q,  Q = [rho_l[N_l, :]]_l,  H (I + 2 M) = -2 [Lambda_l[:, N_l]]_l,
// with M strictly block-triangular over the layers, M[a, b] = Pi_{a-1..b}[N_a, N_b]
// for a > b. By the matrix determinant lemma and det(I + 2M) = 1,
//   det A(x) = det A0 * det(I + K[N, N]),
//   K[(a,i), (b,j)] = 2 [a > b] Pi_{a-1..b}[i, j] - 2 (rho_a A0^{-1})[i, :] Lambda_b[:, j],
// a |N| x |N| determinant over the flipped (layer, mode) pairs, 1 or 2 of
// them for most trajectories of small-angle circuits. Each item's prologue
// builds det A0, A0^{-1} and K over the block's flippable pairs in FP64 (the
// whole CTA, Gauss-Jordan with partial pivoting), then stores K in shared
// memory in the path's precision.
//
// Fallback (the rank-one form): when A0 is singular or ill-conditioned, or a
// trajectory flips more than four pairs of a block, the thread builds A(x)
// by one rank-one update of A0 per flipped mode,
//   A(x) = A0 + sum_l H_l rho_l[N_l, :],
//   H_l  = -2 (Lambda_l[:, N_l] + sum_{l' > l} H_{l'} Pi_{l'-1..l}[N_{l'}, N_l]),
// and factors it (eta x eta LU with partial pivoting).
//
// FP32 error estimate: K is rounded to FP32 and the small determinants are
// formed in FP32; every flipped trajectory s has a first-order bound e_s of its
// rounding error (units of u = 2^-24: the closed forms' input and operation
// roundings, or the LU's pivot proxy). For the K form the roundings of
// distinct small determinants are treated as independent and those of one
// determinant's repeats as equal, so that part of the error of alpha_hat is
// estimated as K u sqrt(n_max sum_s e_s^2) / t, with n_max an upper estimate
// of how many of the t trajectories share one rounded quantity (computed on
// the host from the largest probability that a given flippable pair is
// flipped) and K = 0.5 (calibrated against FP64 on the same trajectories).
// Trajectories through the rank-one form all start from the same FP32 copy of
// A0 and of its update vectors, so their input roundings add up coherently
// (measured: an ill-conditioned A0 of a 12-mode circuit left the FP32 result
// 2.7x its square-root estimate); their bounds are summed linearly,
// u sum_s e_s / t, a first-order worst case. The finalisation turns the sum
// of the two into an estimate of the relative error of p_hat.
// det A0 is FP64, so trajectories without flips carry no error.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "ef_common.cuh"
#include "ef_internal.h"

namespace ef {

__host__ __device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

constexpr int kPartStride = kApproxPartStride;  // per (bitstring, chunk): 5 sums, y0 (2), valid, error sums (2), fallback count
constexpr int kApproxThreads = 128;
constexpr int kMaxKSmall = 4;    // largest |N| evaluated through K

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Dynamic shared memory of one CTA, identical on host and device.
struct ApproxSmem {
    size_t sT, sQr, sGp, sA0[kMaxBlocks], sLeft[kMaxBlocks], sK[kMaxBlocks], aug, lam, yrow, total;
};

__host__ __device__ inline ApproxSmem approx_smem(const ApproxDev& A, int eta_t, size_t csz) {
    ApproxSmem s{};
    size_t off = 0;
    const int k16 = (A.k + 15) & ~15;
    s.sT = off;
    off = al16(off + (size_t)k16 * 4);
    s.sQr = off;  // FP32 ratios (FP32 path)
    off = al16(off + (size_t)k16 * 4);
    s.sGp = off;
    if (A.kform) off = al16(off + (size_t)A.nblocks * A.k * 8);
    int fmax = 0, lnmax = 0;
    for (int B = 0; B < kMaxBlocks; ++B) {
        s.sA0[B] = s.sLeft[B] = s.sK[B] = off;
        if (B >= A.nblocks) continue;
        const ApproxBlockDev& b = A.blk[B];
        s.sA0[B] = off;
        off = al16(off + (size_t)eta_t * eta_t * csz);
        s.sLeft[B] = off;
        off = al16(off + (size_t)b.L * eta_t * b.n * csz);
        s.sK[B] = off;
        if (A.kform) off = al16(off + (size_t)b.f * b.f * csz);
        fmax = b.f > fmax ? b.f : fmax;
        lnmax = b.L * b.n > lnmax ? b.L * b.n : lnmax;
    }
    s.aug = off;
    off = al16(off + (size_t)eta_t * 2 * eta_t * 16);
    s.lam = off;
    if (A.kform) off = al16(off + (size_t)lnmax * eta_t * 16);
    s.yrow = off;
    if (A.kform) off = al16(off + (size_t)fmax * eta_t * 16);
    s.total = off;
    return s;
}

size_t approx_smem_bytes(const ApproxDev& a, int eta_t, bool fp64) {
    return approx_smem(a, eta_t, fp64 ? sizeof(double2) : sizeof(float2)).total;
}

template <typename R> __device__ __forceinline__ R cabs_(cplx_t<R> z) { return sqrt(abs2(z)); }

// det(I + K[N, N]) for |N| = m <= 4 (K row-major with stride f), and for the
// FP32 path a first-order bound of its rounding error in units of u: entries
// of K carry a relative rounding of u; the closed forms add one rounding per
// operation; the 3 x 3 and 4 x 4 LU use the pivot proxy of lu_det_regs.
template <typename R>
__device__ __forceinline__ cplx_t<R> kdet(const cplx_t<R>* __restrict__ K, int f, uint64_t N, int m, R& err) {
    using T = cplx_t<R>;
    int idx[kMaxKSmall];
#pragma unroll
    for (int r = 0; r < kMaxKSmall; ++r) {
        idx[r] = N ? __ffsll((long long)N) - 1 : 0;
        N &= N - 1;
    }
    if (m == 1) {
        const T k = K[idx[0] * f + idx[0]];
        const T d = mk(R(1) + k.x, k.y);
        err = cabs_<R>(k) + cabs_<R>(d);
        return d;
    }
    if (m == 2) {
        const T kii = K[idx[0] * f + idx[0]], kjj = K[idx[1] * f + idx[1]];
        const T b = K[idx[0] * f + idx[1]], c = K[idx[1] * f + idx[0]];
        const T a = mk(R(1) + kii.x, kii.y), e = mk(R(1) + kjj.x, kjj.y);
        const T ae = cmul(a, e), bc = cmul(b, c);
        const T d = mk(ae.x - bc.x, ae.y - bc.y);
        const R na = cabs_<R>(a), ne = cabs_<R>(e), nb = cabs_<R>(b), nc = cabs_<R>(c);
        err = ne * (cabs_<R>(kii) + na) + na * (cabs_<R>(kjj) + ne) + R(3) * na * ne + R(5) * nb * nc + cabs_<R>(d);
        return d;
    }
    T M[kMaxKSmall][kMaxKSmall];
#pragma unroll
    for (int r = 0; r < kMaxKSmall; ++r)
#pragma unroll
        for (int s = 0; s < kMaxKSmall; ++s) {
            T v = mk(R(r == s ? 1 : 0), R(0));
            if (r < m && s < m) {
                const T k = K[idx[r] * f + idx[s]];
                v = mk(v.x + k.x, v.y + k.y);
            }
            M[r][s] = v;
        }
    R er2, zabs2;
    const T d = lu_det_regs<R, kMaxKSmall>(M, er2, zabs2);
    err = sqrt(abs2(d) * er2 + zabs2) + R(m) * cabs_<R>(d);
    return d;
}

// det(I + K[N, N]) for |N| = 1 or 2 (the main loop's cases; no LU code), with
// the same error bound as kdet.
template <typename R>
__device__ __forceinline__ cplx_t<R> kdet12(const cplx_t<R>* __restrict__ K, int f, uint64_t N, int m, R& err) {
    using T = cplx_t<R>;
    const int i0 = __ffsll((long long)N) - 1;
    N &= N - 1;
    const T kii = K[i0 * f + i0];
    const T a = mk(R(1) + kii.x, kii.y);
    if (m == 1) {
        err = cabs_<R>(kii) + cabs_<R>(a);
        return a;
    }
    const int i1 = __ffsll((long long)N) - 1;
    const T kjj = K[i1 * f + i1];
    const T b = K[i0 * f + i1], c = K[i1 * f + i0];
    const T e = mk(R(1) + kjj.x, kjj.y);
    const T ae = cmul(a, e), bc = cmul(b, c);
    const T d = mk(ae.x - bc.x, ae.y - bc.y);
    const R na = cabs_<R>(a), ne = cabs_<R>(e), nb = cabs_<R>(b), nc = cabs_<R>(c);
    err = ne * (cabs_<R>(kii) + na) + na * (cabs_<R>(kjj) + ne) + R(3) * na * ne + R(5) * nb * nc + cabs_<R>(d);
    return d;
}

// det(I + K[N, N]) for |N| = 3 by cofactor expansion, with a first-order
// bound of its FP32 rounding error in units of u (each of the six triple
// products is formed with four roundings from entries carrying one each).
template <typename R>
__device__ __forceinline__ cplx_t<R> kdet3(const cplx_t<R>* __restrict__ K, int f, uint64_t N, R& err) {
    using T = cplx_t<R>;
    int id[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        id[r] = __ffsll((long long)N) - 1;
        N &= N - 1;
    }
    T M[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T k = K[id[r] * f + id[c]];
            M[r][c] = r == c ? mk(R(1) + k.x, k.y) : k;
        }
    const T t0 = cmul(M[0][0], cfms(cmul(M[1][1], M[2][2]), M[1][2], M[2][1]));
    const T t1 = cmul(M[0][1], cfms(cmul(M[1][0], M[2][2]), M[1][2], M[2][0]));
    const T t2 = cmul(M[0][2], cfms(cmul(M[1][0], M[2][1]), M[1][1], M[2][0]));
    const T d = mk(t0.x - t1.x + t2.x, t0.y - t1.y + t2.y);
    R a[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) a[r][c] = cabs_<R>(M[r][c]);
    const R sum = a[0][0] * (a[1][1] * a[2][2] + a[1][2] * a[2][1]) + a[0][1] * (a[1][0] * a[2][2] + a[1][2] * a[2][0]) +
                  a[0][2] * (a[1][0] * a[2][1] + a[1][1] * a[2][0]);
    err = R(7) * sum + cabs_<R>(d);
    return d;
}

// The rank-one form of a block's trajectory minor (see the file comment):
// A(x) = A0 + sum_l H_l rho_l[N_l, :] built from the flipped modes Nl[l - 1]
// of the layers set in lflag, then an eta x eta LU with partial pivoting.
template <typename R, int ETA>
__device__ __noinline__ cplx_t<R> rank_one_det(const ApproxBlockDev& blk, const cplx_t<R>* __restrict__ sA0,
                                                  const cplx_t<R>* __restrict__ sLeft, uint32_t lflag,
                                                  const uint64_t* Nl_in, cplx_t<R> (&hs)[kMaxApproxStored][ETA],
                                                  int (&htag)[kMaxApproxStored], R& er2, R& zabs2) {
    using T = cplx_t<R>;
    const int n = blk.n, Lb = blk.L, ebk = blk.eta;
    const T* P = reinterpret_cast<const T*>(blk.P);
    const T* RC = reinterpret_cast<const T*>(blk.RC);
    T M[ETA][ETA];
#pragma unroll
    for (int i = 0; i < ETA; ++i)
#pragma unroll
        for (int j = 0; j < ETA; ++j) M[i][j] = sA0[i * ETA + j];
    int nst = 0;
    for (int l = Lb; l >= 1; --l) {
        if (!((lflag >> (l - 1)) & 1u)) continue;
        uint64_t Nl = Nl_in[l - 1];
        const bool store = (lflag & ((1u << (l - 1)) - 1u)) != 0;
        const int nabove = nst;  // columns of the layers above l only
        while (Nl) {
            const int i = __ffsll((long long)Nl) - 1;
            Nl &= Nl - 1;
            T h[ETA];
            const T* left = sLeft + (size_t)(l - 1) * ETA * n;
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
            const T* rc = RC + ((size_t)(l - 1) * n + i) * ebk;
#pragma unroll
            for (int c = 0; c < ETA; ++c) {
                if (c < ebk) {
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
    return lu_det_regs<R, ETA>(M, er2, zabs2);
}

// The same for large FP64 minors: rolled loops over a matrix in local memory
// (a few deferred trajectories per thread; unrolled, the FP64 code for
// 9..13 particles spills heavily and takes minutes to compile). Determinant only.
template <typename R, int ETA>
__device__ __noinline__ cplx_t<R> rank_one_det_loop(const ApproxBlockDev& blk, const cplx_t<R>* __restrict__ sA0,
                                                    const cplx_t<R>* __restrict__ sLeft, uint32_t lflag,
                                                    const uint64_t* Nl_in, cplx_t<R> (&hs)[kMaxApproxStored][ETA],
                                                    int (&htag)[kMaxApproxStored]) {
    using T = cplx_t<R>;
    const int n = blk.n, Lb = blk.L, eta = blk.eta;
    const T* P = reinterpret_cast<const T*>(blk.P);
    const T* RC = reinterpret_cast<const T*>(blk.RC);
    T M[ETA][ETA];
#pragma unroll 1
    for (int i = 0; i < eta; ++i)
#pragma unroll 1
        for (int j = 0; j < eta; ++j) M[i][j] = sA0[i * ETA + j];
    int nst = 0;
#pragma unroll 1
    for (int l = Lb; l >= 1; --l) {
        if (!((lflag >> (l - 1)) & 1u)) continue;
        uint64_t Nl = Nl_in[l - 1];
        const bool store = (lflag & ((1u << (l - 1)) - 1u)) != 0;
        const int nabove = nst;
        while (Nl) {
            const int i = __ffsll((long long)Nl) - 1;
            Nl &= Nl - 1;
            T h[ETA];
            const T* left = sLeft + (size_t)(l - 1) * ETA * n;
#pragma unroll 1
            for (int r = 0; r < eta; ++r) {
                T v = left[r * n + i];
                for (int st = 0; st < nabove; ++st) {
                    const int ls = htag[st] >> 8, is = htag[st] & 255;
                    v = cfma(v, hs[st][r], P[(size_t)tri(ls - 1, l) * n * n + (size_t)is * n + i]);
                }
                h[r] = mk(R(-2) * v.x, R(-2) * v.y);
            }
            const T* rc = RC + ((size_t)(l - 1) * n + i) * eta;
#pragma unroll 1
            for (int c = 0; c < eta; ++c) {
                const T v = rc[c];
                for (int r = 0; r < eta; ++r) M[r][c] = cfma(M[r][c], h[r], v);
            }
            if (store && nst < kMaxApproxStored) {
                for (int r = 0; r < eta; ++r) hs[nst][r] = h[r];
                htag[nst] = (l << 8) | i;
                ++nst;
            }
        }
    }
    // LU with partial pivoting (largest |a|^2, lowest row on ties)
    T d = mk(R(1), R(0));
#pragma unroll 1
    for (int k = 0; k < eta; ++k) {
        int p = k;
        R best = abs2(M[k][k]);
        for (int i = k + 1; i < eta; ++i)
            if (abs2(M[i][k]) > best) {
                best = abs2(M[i][k]);
                p = i;
            }
        if (!(best >= min_pivot2(R(0)))) return mk(R(0), R(0));
        if (p != k) {
            d = mk(-d.x, -d.y);
            for (int j = k; j < eta; ++j) {
                const T t = M[k][j];
                M[k][j] = M[p][j];
                M[p][j] = t;
            }
        }
        d = cmul(d, M[k][k]);
        const R ib = R(1) / best;
        const T ip = mk(M[k][k].x * ib, -M[k][k].y * ib);
        for (int i = k + 1; i < eta; ++i) {
            const T l = cmul(M[i][k], ip);
            for (int j = k + 1; j < eta; ++j) M[i][j] = cfms(M[i][j], l, M[k][j]);
        }
    }
    return d;
}

// A trajectory deferred from the main loop// A trajectory deferred from the main loop (more than three flipped pairs in
// a block, or a block whose A0 takes the rank-one form): its flipped pairs
// per block, the product of its sampling ratios and its flip count.
template <typename RQ> struct Deferred {
    uint64_t n[kMaxBlocks];
    RQ rq;
    int nflip;
};

// One trajectory by the general forms, for the deferred trajectories and for
// circuits without the K form: per block det0_B, det0_B det(I + K[N, N]) with
// |N| <= 4, or the rank-one form with an eta x eta LU; returns D = Y - y0, the
// FP32 rounding bound of Y and the number of rank-one minors. Kept out of
// line: the main loop's instruction footprint stays small.
struct GeneralTerm {
    double Dr, Di;
    float es;
    int nfall;
};

template <typename R, int ETA>
__device__ __noinline__ GeneralTerm general_term(const ApproxDev& A, unsigned char* sm_raw, const ApproxSmem& L,
                                                 const double2* s_det0, const float* s_abs0, const int* s_bad,
                                                 const uint32_t (&lflag)[kMaxBlocks], const uint64_t (&Nm)[kMaxBlocks],
                                                 double rq, int nflip, double y0r, double y0i,
                                                 const uint64_t (&N)[kMaxBlocks][kMaxApproxLayers],
                                                 cplx_t<R> (&hs)[kMaxApproxStored][ETA],
                                                 int (&htag)[kMaxApproxStored]) {
    using T = cplx_t<R>;
    constexpr bool kF32 = std::is_same<R, float>::value;
    GeneralTerm out{0.0, 0.0, 0.f, 0};
    double dr = 1.0, di = 0.0;
    float eb[kMaxBlocks] = {}, ab[kMaxBlocks] = {};
    for (int B = 0; B < A.nblocks; ++B) {
        const float a0 = s_abs0[B];
        float e = 0.f, a = a0;
        double2 dd = s_det0[B];
        const int m = __popcll(Nm[B]);
        if (lflag[B] != 0) {
            if (A.kform && !s_bad[B] && m <= kMaxKSmall) {
                if (m > 0) {
                    R err;
                    const T d = kdet<R>(reinterpret_cast<const T*>(sm_raw + L.sK[B]), A.blk[B].f, Nm[B], m, err);
                    dd = cmul(dd, make_double2((double)d.x, (double)d.y));
                    e = a0 * (float)err;
                    a = a0 * (float)cabs_<R>(d);
                }
            } else {
                ++out.nfall;
                R er2, zabs2;
                const T* sA0 = reinterpret_cast<const T*>(sm_raw + L.sA0[B]);
                const T* sLeft = reinterpret_cast<const T*>(sm_raw + L.sLeft[B]);
                T det;
                uint64_t Nl[kMaxApproxLayers] = {};
                uint32_t lf = lflag[B];
                const uint64_t* nl = N[B];
                if (A.kform) {
                    // per-layer flipped modes from the flipped pairs
                    lf = 0;
                    uint64_t pm = Nm[B];
                    while (pm) {
                        const int pp = __ffsll((long long)pm) - 1;
                        pm &= pm - 1;
                        const int v = A.blk[B].pair_lm[pp];
                        Nl[(v >> 8) - 1] |= 1ull << (v & 255);
                        lf |= 1u << ((v >> 8) - 1);
                    }
                    nl = Nl;
                }
                if constexpr (!kF32 && ETA > 8) {
                    det = rank_one_det_loop<R, ETA>(A.blk[B], sA0, sLeft, lf, nl, hs, htag);
                    er2 = zabs2 = R(0);
                } else {
                    det = rank_one_det<R, ETA>(A.blk[B], sA0, sLeft, lf, nl, hs, htag, er2, zabs2);
                }
                dd = make_double2((double)det.x, (double)det.y);
                e = (float)sqrt(abs2(det) * er2 + zabs2);
                a = (float)cabs_<R>(det);
            }
        }
        if (B == 0) eb[0] = e, ab[0] = a;
        else eb[1] = e, ab[1] = a;
        const double t2 = dr * dd.x - di * dd.y;
        di = dr * dd.y + di * dd.x;
        dr = t2;
    }
    const double mag = A.R0 * rq;
    const double2 Y = times_i_pow(make_double2(mag * dr, mag * di), nflip);
    out.Dr = Y.x - y0r;
    out.Di = Y.y - y0i;
    if constexpr (kF32) {
        const float e = A.nblocks == 2 ? eb[0] * ab[1] + eb[1] * ab[0] : eb[0];
        // plus the FP32 rounding of rq (one per flip) and of the products
        out.es = fabsf((float)mag) * e + (float)(nflip + 4) * (float)(fabs(mag) * sqrt(dr * dr + di * di));
    }
    return out;
}

// Resident CTAs per SM the register allocation targets, per instance. Left
// free, the compiler gave the FP32 kernel for five particles 220 registers
// (two CTAs per SM, 5 % slower on the 52-qubit LUCJ workload than at 168);
// the values pin the allocations measured before: FP32 4 / 3 / 2 (255
// registers) CTAs for 1 / 2-5 / 6-13 particles, FP64 3 / 2 / 4 for 1-3 /
// 4-8 / 9-13 (a cap of 3 for the FP32 6-13 kernels made the 64-circuit batch
// 11 % slower).
template <typename R, int ETA>
constexpr int approx_min_ctas() {
    return std::is_same<R, float>::value ? (ETA == 1 ? 4 : ETA <= 5 ? 3 : 1) : (ETA <= 3 ? 3 : ETA <= 8 ? 1 : 4);
}

template <typename R, int ETA>
__global__ void __launch_bounds__(kApproxThreads, approx_min_ctas<R, ETA>())
    k_approx(ApproxDev A, const uint64_t* __restrict__ bits) {
    using T = cplx_t<R>;
    constexpr bool kF32 = std::is_same<R, float>::value;
    using RQ = typename std::conditional<kF32, float, double>::type;
    using DQ = Deferred<RQ>;
    constexpr int NT = kApproxThreads;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ DQ sQ[(NT / 32) * 64];  // per warp: deferred trajectories (at most 63 waiting)
    __shared__ double red[7][NT];
    __shared__ unsigned long long cnt_red[3];
    __shared__ int s_rows[kMaxBlocks][ETA];
    __shared__ double2 s_det0[kMaxBlocks];
    __shared__ float s_abs0[kMaxBlocks];
    __shared__ int s_bad[kMaxBlocks];
    __shared__ double2 s_fac[ETA];
    __shared__ int s_piv;
    __shared__ double s_best, s_cs[ETA];

    const int tid = threadIdx.x;
    const int k = A.k;
    const ApproxSmem L = approx_smem(A, ETA, sizeof(T));
    uint32_t* sT = reinterpret_cast<uint32_t*>(sm_raw + L.sT);
    uint64_t* sGp = reinterpret_cast<uint64_t*>(sm_raw + L.sGp);
    float* sQr = reinterpret_cast<float*>(sm_raw + L.sQr);
    double2* aug = reinterpret_cast<double2*>(sm_raw + L.aug);  // [ETA][2 ETA]
    double2* lam = reinterpret_cast<double2*>(sm_raw + L.lam);  // [L][ETA][n] FP64 Lambda_l rows
    double2* yrow = reinterpret_cast<double2*>(sm_raw + L.yrow);  // [f][ETA] (rho_a A0^{-1}) rows
    const int k16 = (k + 15) & ~15;
    for (int j = tid; j < k16; j += NT) {
        sT[j] = (j < k) ? A.T[j] : 0u;
        if constexpr (kF32) sQr[j] = (j < k) ? A.qratio32[j] : 0.f;
    }
    if (A.kform)
        for (int e = tid; e < A.nblocks * k; e += NT) sGp[e] = A.gpair[e];

    const int64_t n_items = (A.list ? (int64_t)*A.list_count : A.nb) * A.n_chunks;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t bi = item / A.n_chunks;
        const int chunk = (int)(item - bi * A.n_chunks);
        const int64_t b = A.list ? (int64_t)A.list[bi] : bi;
        const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
        double* outp = A.part + ((size_t)b * A.n_chunks + chunk) * kPartStride;

        bool ok = ((w0 & A.inactive0) == 0) && ((w1 & A.inactive1) == 0);
        for (int B = 0; B < A.nblocks; ++B)
            ok = ok && (__popcll(w0 & A.blk[B].mask0) + __popcll(w1 & A.blk[B].mask1) == A.blk[B].eta);
        __syncthreads();  // the previous item's readers of shared memory are done
        if (!ok) {
            if (tid < kPartStride) outp[tid] = 0.0;
            continue;
        }
        if (tid < A.nblocks) {
            int cnt;
            for (int i = 0; i < A.blk[tid].eta; ++i)
                s_rows[tid][i] = nth_row(w0, w1, A.blk[tid].mask0, A.blk[tid].mask1, i, cnt);
        }
        __syncthreads();

        // ---- prologue, block by block: A0 in FP64, det A0 and A0^{-1} by Gauss-Jordan, K
        for (int B = 0; B < A.nblocks; ++B) {
            const ApproxBlockDev& blk = A.blk[B];
            const int n = blk.n, Lb = blk.L, eta = blk.eta, f = blk.f;
            const double2* P64 = blk.P64;
            T* sA0 = reinterpret_cast<T*>(sm_raw + L.sA0[B]);
            T* sLeft = reinterpret_cast<T*>(sm_raw + L.sLeft[B]);
            const double2* PL0 = P64 + (size_t)tri(Lb, 0) * n * n;
            for (int e = tid; e < ETA * 2 * ETA; e += NT) {
                const int i = e / (2 * ETA), j = e - i * 2 * ETA;
                double2 v = make_double2(0.0, 0.0);
                if (i < eta && j < eta) v = PL0[(size_t)s_rows[B][i] * n + blk.cols[j]];
                else if (i < eta && j == eta + i) v = make_double2(1.0, 0.0);
                aug[e] = v;
                if (j < ETA) {
                    T w = mk(R(i == j ? 1 : 0), R(0));
                    if (i < eta && j < eta) w = mk((R)v.x, (R)v.y);
                    else if (i < eta || j < eta) w = mk(R(0), R(0));
                    sA0[i * ETA + j] = w;
                }
            }
            for (int e = tid; e < Lb * ETA * n; e += NT) {
                const int l = e / (ETA * n);
                const int rem = e - l * ETA * n;
                const int i = rem / n, m = rem - i * n;
                double2 v = make_double2(0.0, 0.0);
                if (i < eta) v = P64[(size_t)tri(Lb, l + 1) * n * n + (size_t)s_rows[B][i] * n + m];
                sLeft[e] = mk((R)v.x, (R)v.y);
                if (A.kform) lam[e] = v;
            }
            __syncthreads();
            // ||A0||_1
            if (tid < eta) {
                double cs = 0.0;
                for (int i = 0; i < eta; ++i) cs += sqrt(abs2(aug[i * 2 * ETA + tid]));
                s_cs[tid] = cs;
            }
            if (tid == 0) {
                s_det0[B] = make_double2(1.0, 0.0);
                s_bad[B] = 0;
            }
            __syncthreads();
            double norm_a = 0.0;
            for (int j = 0; j < eta; ++j) norm_a = fmax(norm_a, s_cs[j]);
            for (int kk = 0; kk < eta; ++kk) {
                if (tid < 32) {  // pivot: largest |a_ik|^2 over i >= kk, lowest row on ties
                    double m = -1.0;
                    int p = kk;
                    if (kk + tid < eta) {
                        m = abs2(aug[(kk + tid) * 2 * ETA + kk]);
                        p = kk + tid;
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const double om = __shfl_xor_sync(0xffffffffu, m, off);
                        const int op = __shfl_xor_sync(0xffffffffu, p, off);
                        if (om > m || (om == m && op < p)) {
                            m = om;
                            p = op;
                        }
                    }
                    if (tid == 0) {
                        s_piv = p;
                        s_best = m;
                    }
                }
                __syncthreads();
                const int p = s_piv;
                if (!(s_best >= 2.2250738585072014e-308)) {  // singular (uniform)
                    if (tid == 0) {
                        s_bad[B] = 1;
                        s_det0[B] = make_double2(0.0, 0.0);
                    }
                    break;
                }
                if (p != kk)
                    for (int j = tid; j < 2 * ETA; j += NT) {
                        const double2 t = aug[kk * 2 * ETA + j];
                        aug[kk * 2 * ETA + j] = aug[p * 2 * ETA + j];
                        aug[p * 2 * ETA + j] = t;
                    }
                __syncthreads();
                const double2 piv = aug[kk * 2 * ETA + kk];
                const double ib = 1.0 / s_best;
                const double2 ip = make_double2(piv.x * ib, -piv.y * ib);
                if (tid == 0) {
                    const double2 d = cmul(s_det0[B], piv);
                    s_det0[B] = p != kk ? make_double2(-d.x, -d.y) : d;
                }
                if (tid < eta) s_fac[tid] = aug[tid * 2 * ETA + kk];
                __syncthreads();
                for (int j = tid; j < 2 * ETA; j += NT) aug[kk * 2 * ETA + j] = cmul(aug[kk * 2 * ETA + j], ip);
                __syncthreads();
                for (int e = tid; e < eta * 2 * ETA; e += NT) {
                    const int i = e / (2 * ETA), j = e - i * 2 * ETA;
                    if (i != kk) aug[e] = cfms(aug[e], s_fac[i], aug[kk * 2 * ETA + j]);
                }
                __syncthreads();
            }
            __syncthreads();
            if (!s_bad[B]) {  // condition number ||A0||_1 ||A0^{-1}||_1
                if (tid < eta) {
                    double cs = 0.0;
                    for (int i = 0; i < eta; ++i) cs += sqrt(abs2(aug[i * 2 * ETA + eta + tid]));
                    s_cs[tid] = cs;
                }
                __syncthreads();
                double norm_i = 0.0;
                for (int j = 0; j < eta; ++j) norm_i = fmax(norm_i, s_cs[j]);
                if (tid == 0 && !(norm_a * norm_i <= A.kappa_max)) s_bad[B] = 1;
                __syncthreads();
            }
            if (tid == 0) s_abs0[B] = (float)sqrt(abs2(s_det0[B]));
            if (A.kform && !s_bad[B]) {
                // yrow[p] = rho_a[i, :] A0^{-1} for pair p = (a, i)
                const double2* RC64 = blk.RC64;
                for (int e = tid; e < f * eta; e += NT) {
                    const int pp = e / eta, c = e - pp * eta;
                    const int a = blk.pair_lm[pp] >> 8, i = blk.pair_lm[pp] & 255;
                    const double2* rho = RC64 + ((size_t)(a - 1) * n + i) * eta;
                    double ax = 0.0, ay = 0.0;
                    for (int q = 0; q < eta; ++q) {
                        const double2 x = rho[q], y = aug[q * 2 * ETA + eta + c];
                        ax = fma(x.x, y.x, fma(-x.y, y.y, ax));
                        ay = fma(x.x, y.y, fma(x.y, y.x, ay));
                    }
                    yrow[pp * ETA + c] = make_double2(ax, ay);
                }
                __syncthreads();
                T* sK = reinterpret_cast<T*>(sm_raw + L.sK[B]);
                for (int e = tid; e < f * f; e += NT) {
                    const int pp = e / f, qq = e - pp * f;
                    const int a = blk.pair_lm[pp] >> 8, i = blk.pair_lm[pp] & 255;
                    const int bl = blk.pair_lm[qq] >> 8, j = blk.pair_lm[qq] & 255;
                    double ax = 0.0, ay = 0.0;
                    for (int c = 0; c < eta; ++c) {
                        const double2 x = yrow[pp * ETA + c], y = lam[((size_t)(bl - 1) * ETA + c) * n + j];
                        ax = fma(x.x, y.x, fma(-x.y, y.y, ax));
                        ay = fma(x.x, y.y, fma(x.y, y.x, ay));
                    }
                    ax *= -2.0;
                    ay *= -2.0;
                    if (a > bl) {
                        const double2 mid = P64[(size_t)tri(a - 1, bl) * n * n + (size_t)i * n + j];
                        ax = fma(2.0, mid.x, ax);
                        ay = fma(2.0, mid.y, ay);
                    }
                    sK[e] = mk((R)ax, (R)ay);
                }
            }
            __syncthreads();
        }

        double y0r = A.R0, y0i = 0.0;
        for (int B = 0; B < A.nblocks; ++B) {
            const double2 d = s_det0[B];
            const double nr = y0r * d.x - y0i * d.y;
            y0i = y0r * d.y + y0i * d.x;
            y0r = nr;
        }

        const uint64_t gi = A.gidx ? A.gidx[b] : A.index_base + (uint64_t)b;
        const uint32_t blo = (uint32_t)gi;
        const uint32_t bhi = (uint32_t)(gi >> 32);
        const int64_t s_begin = (int64_t)chunk * A.traj_per_cta;
        const int64_t s_end = min(A.t, s_begin + (int64_t)A.traj_per_cta);
        // Shifted sums of D_s = Y_s - y0 (y0 = the no-flip term). FP64 path,
        // deferred and rank-one-form trajectories: D_s in FP64 (acc). K-form
        // trajectories of the FP32 path: Y_s = y0 g_s with g_s = rq i^nflip prod_B d_B
        // formed in FP32, h_s = g_s - 1 summed in float pairs (its squares in FP32),
        // and the sums of D = y0 h recovered from them in FP64 once per thread.
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        float hs_r = 0.f, hc_r = 0.f, hs_i = 0.f, hc_i = 0.f, h_rr = 0.f, h_ii = 0.f, h_ri = 0.f;
        // per-trajectory rounding bounds: squared, absolute (deferred K-form trajectories) and in
        // units of |y0|^2 (K form inline); linear for the rank-one form (elin)
        float esum = 0.f, gsum = 0.f, elin = 0.f;
        unsigned long long nflips_tot = 0, nlu = 0, nfall = 0;
        uint64_t N[kMaxBlocks][kMaxApproxLayers];
        T hs[kMaxApproxStored][ETA];
        int htag[kMaxApproxStored];
        const int lane = tid & 31, wid = tid >> 5;
        DQ* q = sQ + wid * 64;

        // one trajectory given its flipped modes (rank-one form where needed), added to acc
        auto add_general = [&](const uint32_t (&lflag)[kMaxBlocks], const uint64_t (&Nm)[kMaxBlocks], double rq,
                               int nflip) {
            const GeneralTerm gt = general_term<R, ETA>(A, sm_raw, L, s_det0, s_abs0, s_bad, lflag, Nm, rq, nflip,
                                                        y0r, y0i, N, hs, htag);
            acc[0] += gt.Dr;
            acc[1] += gt.Di;
            acc[2] = fma(gt.Dr, gt.Dr, acc[2]);
            acc[3] = fma(gt.Di, gt.Di, acc[3]);
            acc[4] = fma(gt.Dr, gt.Di, acc[4]);
            if (gt.nfall) elin += gt.es;
            else esum = fmaf(gt.es, gt.es, esum);
            nlu += gt.nfall;
            nfall += gt.nfall;
        };
        // a warp's deferred trajectories, one per lane
        auto drain = [&](int cnt) {
            if (lane < cnt) {
                const DQ e = q[lane];
                uint32_t lf[kMaxBlocks] = {};
                uint64_t nm[kMaxBlocks] = {};
                for (int B = 0; B < A.nblocks; ++B) {
                    nm[B] = e.n[B];
                    lf[B] = e.n[B] ? 1u : 0u;
                }
                add_general(lf, nm, (double)e.rq, e.nflip);
            }
            __syncwarp();
        };

        int qn = 0;  // entries in this warp's queue (the same in every lane)
        for (int64_t s0 = s_begin; s0 < s_end; s0 += NT) {
            const int64_t s = s0 + tid;
            bool defer = false;
            DQ ent{};
            if (s < s_end) {
                // ---- sample the trajectory (Eq. 12 with integer thresholds)
                int nflip = 0;
                RQ rq = RQ(1);
                uint32_t lflag[kMaxBlocks] = {};
                uint64_t Nm[kMaxBlocks] = {};
                // gate j flipped: its ratio and its flips (layer, modes; pairs for the K form)
                auto flip = [&](int j) {
                    ++nflip;
                    if constexpr (kF32) rq *= sQr[j];
                    else rq *= A.qratio[j];
                    if (A.kform) {  // the pair masks alone (zero for a block the gate does not touch)
#pragma unroll
                        for (int B = 0; B < kMaxBlocks; ++B)
                            if (B < A.nblocks) Nm[B] ^= sGp[B * k + j];
                        return;
                    }
#pragma unroll
                    for (int B = 0; B < kMaxBlocks; ++B) {
                        if (B >= A.nblocks) break;
                        const int l = A.glayer[B * k + j];
                        if (l) {
                            const uint32_t bit = 1u << (l - 1);
                            if (A.kform) {
                                Nm[B] ^= sGp[B * k + j];
                            } else {  // per-layer flipped modes for the rank-one form
                                if (!(lflag[B] & bit)) N[B][l - 1] = 0;
                                N[B][l - 1] ^= A.gmodes[B * k + j];
                            }
                            lflag[B] |= bit;
                        }
                    }
                };
                auto hits = [&](const uint4 u, int q4) {
                    const uint4 th = *reinterpret_cast<const uint4*>(sT + 4 * q4);
                    return (uint32_t)(u.x < th.x) | ((uint32_t)(u.y < th.y) << 1) | ((uint32_t)(u.z < th.z) << 2) |
                           ((uint32_t)(u.w < th.w) << 3);
                };
                // four independent Philox blocks at a time (instruction-level parallelism
                // for a chain of dependent multiplies), then their 16 gates' flips in order;
                // the thresholds are padded with zeros to a multiple of 16 gates (no flips)
                const int nq = k16 / 4;
                for (int q4 = 0; q4 < nq; q4 += 4) {
                    const uint4 u0 = philox4x32_10(make_uint4((uint32_t)q4, (uint32_t)s, blo, bhi), A.key0, A.key1);
                    const uint4 u1 =
                        philox4x32_10(make_uint4((uint32_t)q4 + 1u, (uint32_t)s, blo, bhi), A.key0, A.key1);
                    const uint4 u2 =
                        philox4x32_10(make_uint4((uint32_t)q4 + 2u, (uint32_t)s, blo, bhi), A.key0, A.key1);
                    const uint4 u3 =
                        philox4x32_10(make_uint4((uint32_t)q4 + 3u, (uint32_t)s, blo, bhi), A.key0, A.key1);
                    uint32_t hit = hits(u0, q4) | (hits(u1, q4 + 1) << 4) | (hits(u2, q4 + 2) << 8) |
                                   (hits(u3, q4 + 3) << 12);
                    while (hit) {
                        const int w = __ffs(hit) - 1;
                        hit &= hit - 1;
                        flip(4 * q4 + w);
                    }
                }
                nflips_tot += nflip;
                if (nflip > 0) {
                    if (A.kform) {
                        bool small = true;
#pragma unroll
                        for (int B = 0; B < kMaxBlocks; ++B) {
                            if (B >= A.nblocks) break;
                            const int m = __popcll(Nm[B]);
                            small = small && (m == 0 || (!s_bad[B] && m <= 3));
                        }
                        if (small) {
                            // ---- K form inline: d_B = det(I + K[N, N]), |N| <= 3
                            T g = mk(R(1), R(0));
                            R ed[kMaxBlocks] = {}, ad[kMaxBlocks] = {R(1), R(1)};
#pragma unroll
                            for (int B = 0; B < kMaxBlocks; ++B) {
                                if (B >= A.nblocks) break;
                                const int m = __popcll(Nm[B]);
                                if (m == 0) continue;
                                const T* Kb = reinterpret_cast<const T*>(sm_raw + L.sK[B]);
                                R err;
                                const T d = m == 3 ? kdet3<R>(Kb, A.blk[B].f, Nm[B], err)
                                                   : kdet12<R>(Kb, A.blk[B].f, Nm[B], m, err);
                                g = cmul(g, d);
                                ed[B] = err;
                                ad[B] = cabs_<R>(d);
                            }
                            if constexpr (kF32) {
                                // Y_s = y0 rq i^nflip g: accumulate h = rq i^nflip g - 1
                                const float2 qq = make_float2(rq * g.x, rq * g.y);
                                float2 gg = qq;
                                switch (nflip & 3) {
                                    case 1: gg = make_float2(-qq.y, qq.x); break;
                                    case 2: gg = make_float2(-qq.x, -qq.y); break;
                                    case 3: gg = make_float2(qq.y, -qq.x); break;
                                    default: break;
                                }
                                const float hr = gg.x - 1.f, hi = gg.y;
                                {  // error-free additions (Knuth's two-sum), the rounding kept in hc
                                    const float t = hs_r + hr, bp = t - hs_r;
                                    hc_r += (hs_r - (t - bp)) + (hr - bp);
                                    hs_r = t;
                                }
                                {
                                    const float t = hs_i + hi, bp = t - hs_i;
                                    hc_i += (hs_i - (t - bp)) + (hi - bp);
                                    hs_i = t;
                                }
                                h_rr = fmaf(hr, hr, h_rr);
                                h_ii = fmaf(hi, hi, h_ii);
                                h_ri = fmaf(hr, hi, h_ri);
                                const float eg = A.nblocks == 2 ? ed[0] * ad[1] + ed[1] * ad[0] : ed[0];
                                const float es = fabsf(rq) * eg + (float)(nflip + 4) * sqrtf(gg.x * gg.x + gg.y * gg.y);
                                gsum = fmaf(es, es, gsum);
                            } else {
                                const double2 y = cmul(make_double2(y0r, y0i), make_double2(rq * g.x, rq * g.y));
                                const double2 Y = times_i_pow(y, nflip);
                                const double Dr = Y.x - y0r, Di = Y.y - y0i;
                                acc[0] += Dr;
                                acc[1] += Di;
                                acc[2] = fma(Dr, Dr, acc[2]);
                                acc[3] = fma(Di, Di, acc[3]);
                                acc[4] = fma(Dr, Di, acc[4]);
                            }
                        } else {
                            defer = true;
                            for (int B = 0; B < kMaxBlocks; ++B) ent.n[B] = B < A.nblocks ? Nm[B] : 0ull;
                            ent.rq = rq;
                            ent.nflip = nflip;
                        }
                    } else {
                        add_general(lflag, Nm, (double)rq, nflip);
                    }
                }
            }
            if (A.kform) {  // warp queue of deferred trajectories, drained 32 at a time
                const unsigned bal = __ballot_sync(0xffffffffu, defer);
                if (bal) {
                    if (defer) q[qn + __popc(bal & ((1u << lane) - 1u))] = ent;
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn >= 32) {
                        drain(32);
                        if (lane < qn - 32) q[lane] = q[32 + lane];
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
        }
        if (A.kform && qn > 0) drain(qn);
        if constexpr (kF32) {
            // the K-form sums: sum D = y0 sum h; the second moments of D from those of h
            const double sr = (double)hs_r + (double)hc_r, si = (double)hs_i + (double)hc_i;
            const double rr = h_rr, ii = h_ii, ri = h_ri;
            const double a2 = y0r * y0r, b2 = y0i * y0i, ab2 = y0r * y0i;
            acc[0] += y0r * sr - y0i * si;
            acc[1] += y0r * si + y0i * sr;
            acc[2] += a2 * rr - 2.0 * ab2 * ri + b2 * ii;
            acc[3] += a2 * ii + 2.0 * ab2 * ri + b2 * rr;
            acc[4] += (a2 - b2) * ri + ab2 * (rr - ii);
            esum += (float)(y0r * y0r + y0i * y0i) * gsum;
        }

        // ---- deterministic CTA reduction
        for (int e = 0; e < 5; ++e) red[e][tid] = acc[e];
        red[5][tid] = (double)esum;
        red[6][tid] = (double)elin;
        if (tid == 0) cnt_red[0] = cnt_red[1] = cnt_red[2] = 0ull;
        __syncthreads();
        for (int off = NT / 2; off > 0; off >>= 1) {
            if (tid < off)
                for (int e = 0; e < 7; ++e) red[e][tid] += red[e][tid + off];
            __syncthreads();
        }
        atomicAdd(&cnt_red[0], nflips_tot);
        atomicAdd(&cnt_red[1], nlu);
        atomicAdd(&cnt_red[2], nfall);
        __syncthreads();
        if (tid == 0) {
            for (int e = 0; e < 5; ++e) outp[e] = red[e][0];
            outp[5] = y0r;
            outp[6] = y0i;
            outp[7] = 1.0;
            outp[8] = red[5][0];
            outp[9] = (double)cnt_red[2];
            outp[10] = red[6][0];
            atomicAdd(&A.counters[0], cnt_red[0]);
            atomicAdd(&A.counters[1], cnt_red[1] + (unsigned long long)A.nblocks);
            atomicAdd(&A.counters[2], cnt_red[2]);
        }
    }
}

template <typename R, int ETA>
static cudaError_t launch_approx_eta(const ApproxDev& a, const uint64_t* bits, cudaStream_t s) {
    const size_t smem = approx_smem(a, ETA, sizeof(cplx_t<R>)).total;
    cudaError_t e = raise_dynamic_smem((const void*)k_approx<R, ETA>, smem);
    if (e != cudaSuccess) return e;
    k_approx<R, ETA><<<a.grid, kApproxThreads, smem, s>>>(a, bits);
    return cudaGetLastError();
}

// Up to 13 particles per block; for the larger ones the eta x eta matrix of the
// (deferred, rare) rank-one form partly lives in local memory.
template <typename R>
static cudaError_t launch_approx_r(const ApproxDev& a, const uint64_t* bits, int eta, cudaStream_t s) {
    switch (eta) {
        case 1: return launch_approx_eta<R, 1>(a, bits, s);
        case 2: return launch_approx_eta<R, 2>(a, bits, s);
        case 3: return launch_approx_eta<R, 3>(a, bits, s);
        case 4: return launch_approx_eta<R, 4>(a, bits, s);
        case 5: return launch_approx_eta<R, 5>(a, bits, s);
        case 6: return launch_approx_eta<R, 6>(a, bits, s);
        case 7: return launch_approx_eta<R, 7>(a, bits, s);
        case 8: return launch_approx_eta<R, 8>(a, bits, s);
        case 9: return launch_approx_eta<R, 9>(a, bits, s);
        case 10: return launch_approx_eta<R, 10>(a, bits, s);
        case 11: return launch_approx_eta<R, 11>(a, bits, s);
        case 12: return launch_approx_eta<R, 12>(a, bits, s);
        case 13: return launch_approx_eta<R, 13>(a, bits, s);
        default: return cudaErrorInvalidValue;
    }
}

int approx_eta_template(const ApproxDev& a) {
    int eta = 1;
    for (int B = 0; B < a.nblocks; ++B) eta = std::max(eta, a.blk[B].eta);
    return eta;
}

cudaError_t launch_approx(const ApproxDev& a, const uint64_t* bits, bool fp64, cudaStream_t s, LaunchStats& st) {
    if (a.nb <= 0 || a.grid <= 0) return cudaSuccess;
    const int eta = approx_eta_template(a);
    if (eta > (fp64 ? kMaxApproxEta64 : kMaxApproxEta)) return cudaErrorInvalidValue;
    cudaError_t e = fp64 ? launch_approx_r<double>(a, bits, eta, s) : launch_approx_r<float>(a, bits, eta, s);
    st.launches += 1;
    return e;
}

// alpha_hat = Y0 + sum D / t; p_hat = |alpha_hat|^2;
// stderr = 2 sqrt(Var[Re(conj(alpha_hat) Y)] / t) from the shifted sums;
// FP32 path: |delta alpha| ~ (err_coef sqrt(n_max (sum of e_s^2)) + err_lin (sum of the
// rank-one form's e_s)) / t and the estimate of
// the relative error of p_hat, (2 |alpha| |delta alpha| + |delta alpha|^2) / max(p_hat, p_floor).
// Listed mode (the FP64 redo of flagged results) covers the listed bitstrings
// and negates their error estimates.
__global__ void k_approx_finalize(ApproxDev A, double* __restrict__ out, double* __restrict__ se,
                                  double* __restrict__ err, int* __restrict__ append_list,
                                  int* __restrict__ append_count, int listed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t count = listed ? (int64_t)*A.list_count : A.nb;
    if (i >= count) return;
    const int64_t b = listed ? (int64_t)A.list[i] : i;
    const double* p = A.part + (size_t)b * A.n_chunks * kPartStride;
    if (p[7] == 0.0) {
        out[b] = 0.0;
        if (se) se[b] = 0.0;
        if (err) err[b] = 0.0;
        return;
    }
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < A.n_chunks; ++c) {
        for (int e = 0; e < 5; ++e) s[e] += p[(size_t)c * kPartStride + e];
        s[5] += p[(size_t)c * kPartStride + 8];
        s[6] += p[(size_t)c * kPartStride + 10];
    }
    const double t = (double)A.t;
    const double ar = p[5] + s[0] / t, ai = p[6] + s[1] / t;
    const double ph = ar * ar + ai * ai;
    out[b] = ph;
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
    if (listed) {
        if (err) err[b] = -fabs(err[b]);
        return;
    }
    double est = 0.0;
    if (A.err_coef > 0.0) {
        const double da = (A.err_coef * sqrt(A.nmax * s[5]) + A.err_lin * s[6]) / t;
        est = (2.0 * sqrt(ph) * da + da * da) / fmax(ph, A.p_floor);
    }
    if (err) err[b] = est;
    if (append_list && est > A.tol) {
        const int slot = atomicAdd(append_count, 1);
        append_list[slot] = (int)b;
        atomicAdd(&A.counters[3], 1ull);
    }
}

cudaError_t launch_approx_finalize(const ApproxDev& a, double* out, double* stderr_out, double* err_out,
                                   int* append_list, int* append_count, bool listed, cudaStream_t s,
                                   LaunchStats& st) {
    if (a.nb <= 0) return cudaSuccess;
    k_approx_finalize<<<(unsigned)((a.nb + 255) / 256), 256, 0, s>>>(a, out, stderr_out, err_out, append_list,
                                                                    append_count, listed ? 1 : 0);
    st.launches += 1;
    return cudaGetLastError();
}

}  // namespace ef
