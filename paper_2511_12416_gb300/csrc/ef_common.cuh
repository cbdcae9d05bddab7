// Device helpers: complex arithmetic on float2/double2, the Philox4x32-10
// generator and the two small-matrix LU determinant routines used by the
// Exact and Raw Estimate kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ef {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

template <typename R> using cplx_t = typename V2<R>::T;

__host__ __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }

// The fused form is written out so that every kernel that inlines this rounds
// the same way (left to the compiler, which product is fused can depend on the
// surrounding code).
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
    T r;
    r.x = fma(a.x, b.x, -(a.y * b.y));
    r.y = fma(a.x, b.y, a.y * b.x);
    return r;
}
// FP32 cmul as packed FP32x2 instructions (each component rounded exactly as
// cmul's); for kernels with registers to spare (the pairs take a few moves)
__device__ __forceinline__ float2 pcmul(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    const float2 t = __fmul2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x));
    return __ffma2_rn(make_float2(a.x, a.x), b, make_float2(-t.x, t.y));
#else
    return cmul(a, b);
#endif
}
// a - l * p
template <typename T> __device__ __forceinline__ T cfms(T a, T l, T p) {
    T r;
    r.x = fma(-l.x, p.x, fma(l.y, p.y, a.x));
    r.y = fma(-l.x, p.y, fma(-l.y, p.x, a.y));
    return r;
}
// a + l * p
template <typename T> __device__ __forceinline__ T cfma(T a, T l, T p) {
    T r;
    r.x = fma(l.x, p.x, fma(-l.y, p.y, a.x));
    r.y = fma(l.x, p.y, fma(l.y, p.x, a.y));
    return r;
}
template <typename T> __device__ __forceinline__ auto abs2(T a) -> decltype(a.x) {
    return fma(a.x, a.x, a.y * a.y);
}

__device__ __forceinline__ float recip(float m) { return __frcp_rn(m); }
__device__ __forceinline__ double recip(double m) { return 1.0 / m; }
// Smallest |pivot|^2 the eliminations divide by (the smallest normal number):
// below it 1/|p|^2 overflows and a zero component of the pivot turns the
// multipliers into NaN (0 * inf). Such a pivot counts as zero; the error
// proxy's zero-pivot term then covers the determinant, whose size is below
// the rounding error of any entry of its column. Minors of the FP32 path meet
// such pivots when rounding noise stands where an exact zero belongs.
__device__ __forceinline__ float min_pivot2(float) { return 1.17549435e-38f; }
__device__ __forceinline__ double min_pivot2(double) { return 2.2250738585072014e-308; }
// 1/u^2 for the unit roundoff u of the type (2^-24, 2^-53)
__device__ __forceinline__ float inv_u2(float) { return 281474976710656.0f; }
__device__ __forceinline__ double inv_u2(double) { return 81129638414606681695789005144064.0; }
// One pivot's term (k+1) c_k^2 / |u_kk|^2 of the error proxy er2 (units of
// u^2), raised to 1/u^2 (relative error 1) once it exceeds 1/(256 u^2).
template <typename R> __device__ __forceinline__ R pivot_err_term(R t) {
    return t > R(1.0 / 256) * inv_u2(R(0)) ? fmax(t, inv_u2(R(0))) : t;
}

// Stored error term of an FP32 minor: |det|^2 er2 + zabs2 (the absolute
// squared rounding error of the determinant, units of u^2) as a bfloat16
// rounded up, so the stored bound is never below the computed one (at most
// 2^-7 above it). An infinite or undefined term (0 x inf after a vanishing
// pivot) is taken as the largest float, an error too large to bound. The sign
// bit is never set here: a set sign bit (kErrRedone) marks a determinant whose
// value was redone (in float pairs).
__device__ __forceinline__ uint16_t err_term_code(float2 det, float er2, float zabs2) {
    float t = fmaf(fmaf(det.x, det.x, det.y * det.y), er2, zabs2);
    t = t <= 3.0e38f ? t : 3.0e38f;
    const uint32_t u = __float_as_uint(t) & 0x7fffffffu;
    return (uint16_t)((u >> 16) + ((u & 0xffffu) ? 1u : 0u));
}
constexpr uint16_t kErrRedone = 0xbf80u;  // -1 as a bfloat16
__device__ __forceinline__ bool err_redone(uint16_t e) { return (e & 0x8000u) != 0u; }
// the error term (0 for a redone determinant)
__device__ __forceinline__ float err_term_value(uint16_t e) {
    return err_redone(e) ? 0.f : __uint_as_float((uint32_t)e << 16);
}

// multiply by i^ph (ph in 0..3)
__device__ __forceinline__ double2 times_i_pow(double2 a, int ph) {
    switch (ph & 3) {
        case 0: return a;
        case 1: return make_double2(-a.y, a.x);
        case 2: return make_double2(-a.x, -a.y);
        default: return make_double2(a.y, -a.x);
    }
}

// Swap a and b when msk is all ones (no-op when it is zero).
__device__ __forceinline__ void swap_if(float2& a, float2& b, uint32_t msk) {
    const uint32_t dx = (__float_as_uint(a.x) ^ __float_as_uint(b.x)) & msk;
    const uint32_t dy = (__float_as_uint(a.y) ^ __float_as_uint(b.y)) & msk;
    a.x = __uint_as_float(__float_as_uint(a.x) ^ dx);
    a.y = __uint_as_float(__float_as_uint(a.y) ^ dy);
    b.x = __uint_as_float(__float_as_uint(b.x) ^ dx);
    b.y = __uint_as_float(__float_as_uint(b.y) ^ dy);
}
__device__ __forceinline__ void swap_if(double2& a, double2& b, uint32_t msk) {
    const uint64_t m = (uint64_t)msk | ((uint64_t)msk << 32);
    const uint64_t dx = (__double_as_longlong(a.x) ^ __double_as_longlong(b.x)) & m;
    const uint64_t dy = (__double_as_longlong(a.y) ^ __double_as_longlong(b.y)) & m;
    a.x = __longlong_as_double(__double_as_longlong(a.x) ^ dx);
    a.y = __longlong_as_double(__double_as_longlong(a.y) ^ dy);
    b.x = __longlong_as_double(__double_as_longlong(b.x) ^ dx);
    b.y = __longlong_as_double(__double_as_longlong(b.y) ^ dy);
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds; each multiplies counter words 0 and 2 by
// fixed odd constants, keeps the high and low product halves and mixes the
// high halves with the other words and the key; the key advances by two Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ---------------------------------------------------------------- bitstrings
// Local row indices (ascending) of the set bits of (w0, w1) inside a block
// given by its global mode mask. Returns false unless there are exactly N.
template <int N>
__device__ __forceinline__ bool decode_rows(uint64_t w0, uint64_t w1, uint64_t m0, uint64_t m1,
                                            int (&rows)[N]) {
    w0 &= m0;
    w1 &= m1;
    const int base1 = __popcll(m0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        int r = -1;
        if (w0) {
            const int m = __ffsll((long long)w0) - 1;
            w0 &= w0 - 1;
            r = __popcll(m0 & ((1ull << m) - 1ull));
        } else if (w1) {
            const int m = __ffsll((long long)w1) - 1;
            w1 &= w1 - 1;
            r = base1 + __popcll(m1 & ((1ull << m) - 1ull));
        }
        rows[i] = r;
    }
    bool ok = (w0 == 0) && (w1 == 0);
#pragma unroll
    for (int i = 0; i < N; ++i) ok = ok && rows[i] >= 0;
    return ok;
}

// The local row index of the r-th set bit (r < popcount) of (w0,w1) & mask,
// or -1; also returns the popcount through cnt.
__device__ __forceinline__ int nth_row(uint64_t w0, uint64_t w1, uint64_t m0, uint64_t m1, int r,
                                       int& cnt) {
    w0 &= m0;
    w1 &= m1;
    const int c0 = __popcll(w0);
    cnt = c0 + __popcll(w1);
    if (r < 0 || r >= cnt) return -1;
    uint64_t w = (r < c0) ? w0 : w1;
    int rr = (r < c0) ? r : r - c0;
    for (int i = 0; i < rr; ++i) w &= w - 1;
    const int m = __ffsll((long long)w) - 1;
    if (r < c0) return __popcll(m0 & ((1ull << m) - 1ull));
    return __popcll(m0) + __popcll(m1 & ((1ull << m) - 1ull));
}

// ---------------------------------------------------------------- LU determinants
// Thread-per-minor LU with partial pivoting (largest |a|^2 in the column,
// lowest current row on ties) on an N x N matrix in registers.
//
// Besides the determinant it returns a rounding-error proxy for the FP32
// path. Pivot u_kk is formed by k+1 rounded updates of entries no larger than
// the original column's largest entry c_k, so its relative error is about
// sqrt(k+1) u c_k / |u_kk|; the determinant's relative error squared is then
// er2 = sum_k (k+1) c_k^2 / |u_kk|^2 (in units of u^2). A zero pivot (|u_kk|^2
// below the smallest normal number) leaves det ~ 0 with an absolute error of about
// sqrt(k+1) u c_k prod_{j != k} |u_jj|; zabs2 is the square of that (0 when no
// pivot vanished). A pivot whose own term puts its relative error above 1/16 is
// taken for rounding noise (the minor is singular up to rounding; the backward
// error of the elimination allows such a pivot up to ~n * growth * u * c_k,
// several times its term, and one of a singular 7x7 minor sat at 0.27): its
// term becomes 1/u^2, a relative error of 1 for the determinant. The elimination steps are a
// compile-time recursion so every matrix index is a constant and the matrix
// stays in registers.
// Rows K+1.. minus l_i times the pivot row K, l_i = A[i][K] / pivot (ip = 1/pivot).
// In FP32 on sm_100+ each complex update a - l p is two packed FP32x2 FMAs,
// (a.x, a.y) + (-l.x, -l.x)(p.x, p.y) + (l.y, -l.y)(p.y, p.x).
template <typename R, int N, int K>
__device__ __forceinline__ void eliminate(cplx_t<R> (&A)[N][N], cplx_t<R> ip) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    if constexpr (std::is_same<R, float>::value) {
        float2 psw[N];
#pragma unroll
        for (int j = K + 1; j < N; ++j) psw[j] = make_float2(A[K][j].y, A[K][j].x);
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const float2 l = cmul(A[i][K], ip);
            const float2 nl = make_float2(-l.x, -l.x);
            const float2 ly = make_float2(l.y, -l.y);
#pragma unroll
            for (int j = K + 1; j < N; ++j) A[i][j] = __ffma2_rn(ly, psw[j], __ffma2_rn(nl, A[K][j], A[i][j]));
        }
    } else
#endif
    {
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const cplx_t<R> l = cmul(A[i][K], ip);
#pragma unroll
            for (int j = K + 1; j < N; ++j) A[i][j] = cfms(A[i][j], l, A[K][j]);
        }
    }
}

template <typename R, int N, int K>
__device__ __forceinline__ void lu_step(cplx_t<R> (&A)[N][N], const R (&cm2)[N], cplx_t<R>& d, bool& odd,
                                        R& er2, R& pz, R& zc, int& nzero) {
    if constexpr (K < N) {
        using T = cplx_t<R>;
        R best = abs2(A[K][K]);
        int p = K;
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const R m = abs2(A[i][K]);
            const bool gt = m > best;
            best = gt ? m : best;
            p = gt ? i : p;
        }
        odd ^= (p != K);
        // exchange rows K and p: gather the pivot row by selects, then put the
        // old row K into slot p (columns >= K only; the rest is never read again)
        T prow[N];
#pragma unroll
        for (int j = K; j < N; ++j) prow[j] = A[K][j];
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = K; j < N; ++j) prow[j] = s ? A[i][j] : prow[j];
        }
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = K; j < N; ++j) A[i][j] = s ? A[K][j] : A[i][j];
        }
#pragma unroll
        for (int j = K; j < N; ++j) A[K][j] = prow[j];
        const T piv = A[K][K];
        d = cmul(d, piv);
        const bool nz = best >= min_pivot2(R(0));
        const R inv = nz ? recip(best) : R(0);
        er2 += pivot_err_term(R(K + 1) * cm2[K] * inv);
        pz *= nz ? best : R(1);
        zc = nz ? zc : R(K + 1) * cm2[K];
        nzero += nz ? 0 : 1;
        const T ip = mk(piv.x * inv, -piv.y * inv);
        eliminate<R, N, K>(A, ip);
        lu_step<R, N, K + 1>(A, cm2, d, odd, er2, pz, zc, nzero);
    }
}

template <typename R, int N>
__device__ __forceinline__ cplx_t<R> lu_det_regs(cplx_t<R> (&A)[N][N], R& er2, R& zabs2) {
    using T = cplx_t<R>;
    R cm2[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        R m = abs2(A[0][j]);
#pragma unroll
        for (int i = 1; i < N; ++i) m = fmax(m, abs2(A[i][j]));
        cm2[j] = m;
    }
    T d = mk(R(1), R(0));
    bool odd = false;
    R pz = R(1), zc = R(0);
    int nzero = 0;
    er2 = R(0);
    lu_step<R, N, 0>(A, cm2, d, odd, er2, pz, zc, nzero);
    zabs2 = (nzero == 1) ? zc * pz : R(0);
    return odd ? mk(-d.x, -d.y) : d;
}

// The same elimination without the rounding-error proxy: for results that
// are final (FP64) rather than estimated.
template <typename R, int N, int K>
__device__ __forceinline__ void lu_step_plain(cplx_t<R> (&A)[N][N], cplx_t<R>& d, bool& odd) {
    if constexpr (K < N) {
        using T = cplx_t<R>;
        R best = abs2(A[K][K]);
        int p = K;
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const R m = abs2(A[i][K]);
            const bool gt = m > best;
            best = gt ? m : best;
            p = gt ? i : p;
        }
        odd ^= (p != K);
        T prow[N];
#pragma unroll
        for (int j = K; j < N; ++j) prow[j] = A[K][j];
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = K; j < N; ++j) prow[j] = s ? A[i][j] : prow[j];
        }
#pragma unroll
        for (int i = K + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = K; j < N; ++j) A[i][j] = s ? A[K][j] : A[i][j];
        }
#pragma unroll
        for (int j = K; j < N; ++j) A[K][j] = prow[j];
        const T piv = A[K][K];
        d = cmul(d, piv);
        const R inv = best >= min_pivot2(R(0)) ? recip(best) : R(0);
        const T ip = mk(piv.x * inv, -piv.y * inv);
        eliminate<R, N, K>(A, ip);
        lu_step_plain<R, N, K + 1>(A, d, odd);
    }
}

template <typename R, int N>
__device__ __forceinline__ cplx_t<R> lu_det_plain(cplx_t<R> (&A)[N][N]) {
    cplx_t<R> d = mk(R(1), R(0));
    bool odd = false;
    lu_step_plain<R, N, 0>(A, d, odd);
    return odd ? mk(-d.x, -d.y) : d;
}

// Warp-row LU: a group of G lanes (G a power of two, 1 < G <= 32) holds one
// eta x eta minor, lane r of the group owning row r (rows >= eta are padding).
// The rows never move: at step k the group finds the pivot row p (largest
// |a_rk|^2 among rows not yet used, lowest r on ties) by shuffles, broadcasts
// its remaining entries and every other unused row eliminates against it.
// The permutation's sign is the parity of the number of unused rows below p
// at each step. All 32 lanes of the warp must call this with the same eta.
// er2 and zabs2 are the rounding-error proxies of lu_det_regs.
template <typename R, int G>
__device__ __forceinline__ cplx_t<R> lu_det_rows(cplx_t<R> (&row)[G], int r, int eta, R& er2, R& zabs2) {
    using T = cplx_t<R>;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    bool done = (r >= eta);
    T d = mk(R(1), R(0));
    int inv = 0;
    R pz = R(1), zc = R(0);
    int nzero = 0;
    er2 = R(0);
    // largest |entry|^2 of every original column
    R cm2[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        R cm = (done || j >= eta) ? R(0) : abs2(row[j]);
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) cm = fmax(cm, __shfl_xor_sync(full, cm, off, G));
        cm2[j] = cm;
    }
#pragma unroll
    for (int k = 0; k < G; ++k) {
        if (k >= eta) break;
        const R cm = cm2[k];
        R mag = done ? R(-1) : abs2(row[k]);
        int idx = r;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            const R om = __shfl_xor_sync(full, mag, off, G);
            const int oi = __shfl_xor_sync(full, idx, off, G);
            if (om > mag || (om == mag && oi < idx)) {
                mag = om;
                idx = oi;
            }
        }
        const int p = idx;
        const unsigned act = (__ballot_sync(full, !done) >> gbase) & gmask;
        inv += __popc(act & ((1u << p) - 1u));
        T piv;
        piv.x = __shfl_sync(full, row[k].x, p, G);
        piv.y = __shfl_sync(full, row[k].y, p, G);
        const R best = mag;
        d = cmul(d, piv);
        const bool nz = best >= min_pivot2(R(0));
        const R invm = nz ? recip(best) : R(0);
        er2 += pivot_err_term(R(k + 1) * cm * invm);
        pz *= nz ? best : R(1);
        zc = nz ? zc : R(k + 1) * cm;
        nzero += nz ? 0 : 1;
        const T ip = mk(piv.x * invm, -piv.y * invm);
        const bool upd = !done && (r != p);
        const T l = cmul(row[k], ip);
#pragma unroll
        for (int j = k + 1; j < G; ++j) {
            if (j >= eta) break;
            T pj;
            pj.x = __shfl_sync(full, row[j].x, p, G);
            pj.y = __shfl_sync(full, row[j].y, p, G);
            if (upd) row[j] = cfms(row[j], l, pj);
        }
        if (r == p) done = true;
    }
    zabs2 = (nzero == 1) ? zc * pz : R(0);
    return (inv & 1) ? mk(-d.x, -d.y) : d;
}

}  // namespace ef
