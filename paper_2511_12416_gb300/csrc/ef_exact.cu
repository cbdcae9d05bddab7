// Exact algorithm (Section III-B, Eqs. 8-9) on the GPU.
//
// The circuit's modes split into at most two independent blocks (modes joined
// by Givens rotations; controlled-phase gates are diagonal and never join
// them). For a trajectory x the mode matrix is block diagonal, so the minor's
// determinant is the product of the blocks' minors. Inside a block the
// trajectory enters only through its flip pattern: D_{x_j} = D_0 W_j with
// W_j = diag(-1 on the gate's modes)^{x_j} (Section IV-B, Eqs. 15-16), so the
// block's matrix is U(x) = T_L W_L(x) ... T_1 W_1(x) S_0 with W_l(x) the
// product of the layer's W_j: only which modes flip in which layer matters.
// Patterns form a GF(2) vector space; each block enumerates the 2^r patterns
// once instead of the 2^{k_B} bit vectors, and the host folds the branch
// weights w(x) onto patterns. Per block:
//
//   1. k_build_branches : U_B(z)[:, C_B] for every pattern z (dense products, FP64 or
//                         float pairs);
//   2. k_exact_lu_*     : det U_B(z)[R_B(b), C_B] (Eq. 3) for every (pattern, bitstring),
//                         LU with partial pivoting, plus a rounding-error proxy
//                         (the FP32 kernels are in ef_lu32.cu);
//   3. k_exact_combine  : amp(b) = sum_{x_sh} w_sh(x_sh) prod_B A_B(x_sh) with
//                         A_B(x_sh) = sum_{z local} Omega_B(z) det_B(z ^ s_B(x_sh)),
//                         p(b) = |amp|^2, and the FP32 path's error estimate.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "ef_common.cuh"
#include "ef_internal.h"

namespace ef {

cudaError_t raise_dynamic_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[{dev, kernel}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// Streaming multiprocessors of the current device (queried once per device).
// It only sizes grids: if the query fails, the launch that follows fails too,
// so the fallback value merely keeps the grid arithmetic defined.
int sm_count() {
    constexpr int kFallback = 128;
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kFallback;
    if (cached[dev] <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = kFallback;
        cached[dev] = v;
    }
    return cached[dev];
}

// ---- float-pair ("double-float") arithmetic for the branch-matrix builder,
// the transforms over FP32 determinants and the redo of listed determinants:
// a value is hi + lo with |lo| <= ulp(hi)/2, about 48 bits.
// Sums use the error-free two-sum (Knuth) and products the FMA residual
// (Dekker's product with a fused multiply-add), each renormalised.

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 ff_add(float2 x, float2 y) {
    const float2 s = two_sum(x.x, y.x);
    return quick_two_sum(s.x, s.y + (x.y + y.y));
}
__device__ __forceinline__ float2 ff_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 ff_mul(float2 x, float2 y) {
    const float p = x.x * y.x;
    const float e = fmaf(x.x, y.y, fmaf(x.y, y.x, fmaf(x.x, y.x, -p)));
    return quick_two_sum(p, e);
}
// Complex float pairs as float4 (re hi, im hi, re lo, im lo): the leading
// parts form one FP32 complex and the trailing parts another, so the real and
// imaginary float-pair operations run as packed FP32x2 instructions, one
// instruction for both (each component is rounded exactly as the scalar
// operation would be).
__device__ __forceinline__ float2 cf_re(float4 v) { return make_float2(v.x, v.z); }
__device__ __forceinline__ float2 cf_im(float4 v) { return make_float2(v.y, v.w); }
__device__ __forceinline__ float2 cf_hi(float4 v) { return make_float2(v.x, v.y); }  // leading parts (FP32 complex)
__device__ __forceinline__ float4 cf_make(float2 re, float2 im) { return make_float4(re.x, im.x, re.y, im.y); }
__device__ __forceinline__ float4 cf_from_f(float2 z) { return make_float4(z.x, z.y, 0.f, 0.f); }

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
__device__ __forceinline__ float2 p2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#else
__device__ __forceinline__ float2 p2_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 p2_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 p2_mul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 p2_fma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#endif

// Two float-pair additions at once: ff_add on (xh.x, xl.x) + (yh.x, yl.x) and
// on the .y components, in ff_add's order of operations.
__device__ __forceinline__ float4 cf_add(float4 a, float4 b) {
    const float2 ah = make_float2(a.x, a.y), al = make_float2(a.z, a.w);
    const float2 bh = make_float2(b.x, b.y), bl = make_float2(b.z, b.w);
    const float2 s = p2_add(ah, bh);
    const float2 bb = p2_sub(s, ah);
    const float2 e = p2_add(p2_sub(ah, p2_sub(s, bb)), p2_sub(bh, bb));
    const float2 t = p2_add(e, p2_add(al, bl));
    const float2 r = p2_add(s, t);
    const float2 lo = p2_sub(t, p2_sub(r, s));
    return make_float4(r.x, r.y, lo.x, lo.y);
}
__device__ __forceinline__ float4 cf_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 cf_sub(float4 a, float4 b) { return cf_add(a, cf_neg(b)); }
// Two float-pair products at once (ff_mul's order of operations).
__device__ __forceinline__ float4 cf_mul2(float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 p = p2_mul(xh, yh);
    const float2 e = p2_fma(xh, yl, p2_fma(xl, yh, p2_fma(xh, yh, make_float2(-p.x, -p.y))));
    const float2 s = p2_add(p, e);
    const float2 lo = p2_sub(e, p2_sub(s, p));
    return make_float4(s.x, s.y, lo.x, lo.y);
}
// complex product: (ar br, ar bi) + (-ai bi, ai br), as the scalar
// ff_add(ff_mul(ar, br), -ff_mul(ai, bi)) and ff_add(ff_mul(ar, bi), ff_mul(ai, br))
__device__ __forceinline__ float4 cf_mul(float4 a, float4 b) {
    const float4 p1 = cf_mul2(make_float2(a.x, a.x), make_float2(a.z, a.z), make_float2(b.x, b.y),
                              make_float2(b.z, b.w));
    const float4 p2 = cf_mul2(make_float2(-a.y, a.y), make_float2(-a.w, a.w), make_float2(b.y, b.x),
                              make_float2(b.w, b.z));
    return cf_add(p1, p2);
}

// ---------------------------------------------------------------- 1. builder

// Blocks B0 and B1 (blockIdx.y) in one launch: each is mostly latency at this
// size, so two launches cost about twice one.
//
// With FP32 outputs wanted (every precision but EF_PREC_FP64) and at most
// kBuildFFModes modes, the products run in float pairs (about 48 bits) on the
// FP32 pipes instead of FP64 (an FP64 instruction costs a warp about 64 cycles
// of its sub-partition's FP64 unit): M32 gets the leading parts, ML32 the
// trailing ones, M64 their sum (used only by the whole-bitstring FP64 redo).
// The plain FP64 form keeps FP64 products.
constexpr int kBuildFFModes = 64;

__device__ __forceinline__ float4 cf_of_d(double2 a) {
    const float rh = (float)a.x, ih = (float)a.y;
    return make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
}

__global__ void __launch_bounds__(128) k_build_branches(ExactBlockDev B0, ExactBlockDev B1, int want32) {
    cudaGridDependencySynchronize();  // see launch_pdl
    extern __shared__ double2 smb[];
    const ExactBlockDev& B = blockIdx.y ? B1 : B0;
    const int n = B.n, eta = B.eta, ne = n * eta;
    const uint32_t ny = 1u << B.r;
    if (want32 && n <= kBuildFFModes) {
        float4* cur = reinterpret_cast<float4*>(smb);
        float4* nxt = cur + ne;
        float4* Tf = nxt + ne;
        int* sgn = reinterpret_cast<int*>(Tf + (size_t)n * n);
        for (uint32_t z = blockIdx.x; z < ny; z += gridDim.x) {
            for (int e = threadIdx.x; e < ne; e += blockDim.x) cur[e] = cf_of_d(B.S0C[e]);
            for (int l = 0; l < B.L; ++l) {
                for (int m = threadIdx.x; m < n; m += blockDim.x) sgn[m] = __popc(z & B.F[l * n + m]) & 1;
                const double2* T = B.T + (size_t)l * n * n;
                for (int e = threadIdx.x; e < n * n; e += blockDim.x) Tf[e] = cf_of_d(T[e]);
                __syncthreads();
                for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                    const int i = e / eta, c = e - i * eta;
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int m = 0; m < n; ++m) {
                        const float4 x = cur[m * eta + c];
                        acc = cf_add(acc, cf_mul(Tf[i * n + m], sgn[m] ? cf_neg(x) : x));
                    }
                    nxt[e] = acc;
                }
                __syncthreads();
                float4* tmp = cur;
                cur = nxt;
                nxt = tmp;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < ne; e += blockDim.x) {
                const float4 v = cur[e];
                const size_t o = (size_t)z * ne + e;
                B.M32[o] = make_float2(v.x, v.y);
                B.ML32[o] = make_float2(v.z, v.w);
                B.M64[o] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
            }
            __syncthreads();
        }
        return;
    }
    double2* bufA = smb;
    double2* bufB = smb + ne;
    int* sgn = reinterpret_cast<int*>(smb + 2 * ne);
    for (uint32_t z = blockIdx.x; z < ny; z += gridDim.x) {
        double2* cur = bufA;
        double2* nxt = bufB;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) cur[e] = B.S0C[e];
        for (int l = 0; l < B.L; ++l) {
            for (int m = threadIdx.x; m < n; m += blockDim.x) sgn[m] = __popc(z & B.F[l * n + m]) & 1;
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
        double2* o64 = B.M64 + (size_t)z * ne;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const double2 v = cur[e];
            o64[e] = v;
            if (want32) {
                const float rh = (float)v.x, ih = (float)v.y;
                B.M32[(size_t)z * ne + e] = make_float2(rh, ih);
                B.ML32[(size_t)z * ne + e] = make_float2((float)(v.x - (double)rh), (float)(v.y - (double)ih));
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_build_branches(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk, bool want32,
                                  cudaStream_t s, LaunchStats& st) {
    if (nblk < 1 || nblk > 2) return cudaErrorInvalidValue;
    size_t smem = 0;
    uint32_t ny = 1;
    for (int i = 0; i < nblk; ++i) {
        const ExactBlockDev& b = i ? b1 : b0;
        smem = std::max(smem, (size_t)2 * b.n * b.eta * sizeof(double2) + (size_t)b.n * sizeof(int));
        if (want32 && b.n <= kBuildFFModes)  // float-pair path: the layer's T staged as float pairs too
            smem = std::max(smem, (size_t)(2 * b.n * b.eta + b.n * b.n) * sizeof(float4) + (size_t)b.n * sizeof(int));
        ny = std::max(ny, 1u << b.r);
    }
    cudaError_t e = raise_dynamic_smem((const void*)k_build_branches, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(std::min<uint32_t>(ny, (uint32_t)sm_count() * 16u), (unsigned)nblk);
    const cudaError_t le = launch_pdl(k_build_branches, grid, dim3(128), smem, s, b0, nblk == 2 ? b1 : b0, want32 ? 1 : 0);
    if (le != cudaSuccess) return le;
    st.launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- 2b. FP64, thread per minor
// Thread <-> (pattern, bitstring) work item, consecutive threads on
// consecutive bitstrings of one pattern; the minor is gathered from the FP64
// branch matrices in L2. Used for eta <= 8 (the FP64 pipe, not the register
// file, bounds it; the compiler may keep part of the matrix in local memory).

template <int ETA>
__global__ void __launch_bounds__(128) k_exact_lu_f64t(ExactBlockDev B, const uint64_t* __restrict__ bits,
                                                       int64_t nb, const int* __restrict__ list,
                                                       const int* __restrict__ list_count, int64_t stride) {
    cudaGridDependencySynchronize();  // see launch_pdl
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    const int64_t total = count << B.r;
    const int n = B.n;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < total;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = item / count;
        const int64_t pos = item - z * count;
        const int64_t b = list ? (int64_t)list[pos] : pos;
        int rows[ETA];
        double2 res = make_double2(0.0, 0.0);
        if (decode_rows<ETA>(bits[2 * b], bits[2 * b + 1], B.mask0, B.mask1, rows)) {
            const double2* Mz = B.M64 + (size_t)z * n * ETA;
            double2 A[ETA][ETA];
#pragma unroll
            for (int i = 0; i < ETA; ++i)
#pragma unroll
                for (int j = 0; j < ETA; ++j) A[i][j] = Mz[rows[i] * ETA + j];
            res = lu_det_plain<double, ETA>(A);
        }
        B.D64[dix(pos, (uint32_t)z, B.r)] = res;
    }
}

template <int ETA>
static cudaError_t launch_f64t_eta(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                   const int* list_count, int64_t stride, cudaStream_t s) {
    // list mode: the list is usually short or empty, so a small grid strides over it
    const int64_t items = (list ? stride : nb) << b.r;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((items + 127) / 128, list ? sm_count() : sm_count() * 32));
    const cudaError_t le = launch_pdl(k_exact_lu_f64t<ETA>, dim3((unsigned)blocks), dim3(128), 0, s, b, bits, nb, list, list_count, stride);
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- 2c. warp-row LU (FP64, or FP32 for large eta)
// A group of G lanes handles one (bitstring, chunk of patterns) work item;
// lane r holds row r of each minor. Work items are visited warp-uniformly in
// a grid-stride loop; in list mode the bitstrings are list[0..*list_count)
// (the results the FP32 path flagged) and determinants go to
// D[pattern][list position] (row stride `stride`).

template <typename R, int G>
__global__ void __launch_bounds__(256) k_exact_lu_rows(ExactBlockDev B, const uint64_t* __restrict__ bits,
                                                       int64_t nb, const int* __restrict__ list,
                                                       const int* __restrict__ list_count, int64_t stride,
                                                       const cplx_t<R>* __restrict__ M) {
    using T = cplx_t<R>;
    const int lane = threadIdx.x & 31;
    const int r = lane & (G - 1);
    constexpr int GPW = 32 / G;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    const int Y = 1 << B.c_log2;
    const int64_t total = count * (int64_t)B.n_chunks;
    const int n = B.n, eta = B.eta;
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
        for (int t = 0; t < Y; ++t) {
            const size_t z = (size_t)chunk * Y + t;
            T rowv[G];
            const T* src = M + (z * n + (size_t)(row_idx < 0 ? 0 : row_idx)) * eta;
            const bool live = ok && r < eta;
#pragma unroll
            for (int j = 0; j < G; ++j) rowv[j] = (live && j < eta) ? src[j] : mk(R(0), R(0));
            R er2, zabs2;
            const T det = lu_det_rows<R, G>(rowv, r, eta, er2, zabs2);
            if (valid && r == 0) {
                if constexpr (std::is_same<R, double>::value)
                    B.D64[dix(pos, (uint32_t)z, B.r)] = ok ? det : make_double2(0.0, 0.0);
                else {
                    const size_t o = dix(pos, (uint32_t)z, B.r);
                    B.D32[o] = ok ? det : make_float2(0.f, 0.f);
                    B.E32[o] = ok ? err_term_code(det, er2, zabs2) : (uint16_t)0;
                }
            }
        }
    }
}

template <typename R, int G>
static cudaError_t launch_rows_g(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, int64_t stride, const void* M, cudaStream_t s) {
    const int64_t items = (list ? stride : nb) * (int64_t)b.n_chunks;
    const int64_t warps = (items + (32 / G) - 1) / (32 / G);
    int64_t blocks = (warps + 7) / 8;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
    k_exact_lu_rows<R, G><<<(unsigned)blocks, 256, 0, s>>>(b, bits, nb, list, list_count, stride,
                                                          reinterpret_cast<const cplx_t<R>*>(M));
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_rows_r(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, int64_t stride, const void* M, cudaStream_t s) {
    if (b.eta <= 2) return launch_rows_g<R, 2>(b, bits, nb, list, list_count, stride, M, s);
    if (b.eta <= 4) return launch_rows_g<R, 4>(b, bits, nb, list, list_count, stride, M, s);
    if (b.eta <= 8) return launch_rows_g<R, 8>(b, bits, nb, list, list_count, stride, M, s);
    if (b.eta <= 16) return launch_rows_g<R, 16>(b, bits, nb, list, list_count, stride, M, s);
    return launch_rows_g<R, 32>(b, bits, nb, list, list_count, stride, M, s);
}

cudaError_t launch_exact_lu_rows(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                 const int* list_count, int64_t cap, bool fp64, cudaStream_t s, LaunchStats& st) {
    if ((list ? cap : nb) <= 0) return cudaSuccess;
    if (b.eta > kMaxEtaRows) return cudaErrorInvalidValue;
    cudaError_t e = fp64 ? launch_rows_r<double>(b, bits, nb, list, list_count, cap, b.M64, s)
                         : launch_rows_r<float>(b, bits, nb, list, list_count, cap, b.M32, s);
    st.launches += 1;
    if (!list) st.executed_lus += nb * ((int64_t)1 << b.r);
    return e;
}

cudaError_t launch_exact_lu_f64(const ExactBlockDev& b, const uint64_t* bits, int64_t nb, const int* list,
                                const int* list_count, int64_t cap, cudaStream_t s, LaunchStats& st) {
    if ((list ? cap : nb) <= 0) return cudaSuccess;
    cudaError_t e;
    switch (b.eta) {
        case 1: e = launch_f64t_eta<1>(b, bits, nb, list, list_count, cap, s); break;
        case 2: e = launch_f64t_eta<2>(b, bits, nb, list, list_count, cap, s); break;
        case 3: e = launch_f64t_eta<3>(b, bits, nb, list, list_count, cap, s); break;
        case 4: e = launch_f64t_eta<4>(b, bits, nb, list, list_count, cap, s); break;
        case 5: e = launch_f64t_eta<5>(b, bits, nb, list, list_count, cap, s); break;
        case 6: e = launch_f64t_eta<6>(b, bits, nb, list, list_count, cap, s); break;
        case 7: e = launch_f64t_eta<7>(b, bits, nb, list, list_count, cap, s); break;
        case 8: e = launch_f64t_eta<8>(b, bits, nb, list, list_count, cap, s); break;
        default: return launch_exact_lu_rows(b, bits, nb, list, list_count, cap, true, s, st);
    }
    st.launches += 1;
    if (!list) st.executed_lus += nb * ((int64_t)1 << b.r);
    return e;
}

// ---------------------------------------------------------------- 3. combine
// One CTA per bitstring. Phase 1 (FP64): A_B(x_sh) for every shared bit
// vector and amp = sum w_sh A_0 A_1. Phase 2 (FP32 path only): the error
// estimate. Each determinant det_B(z) enters amp with the coefficient
// C_B(z) = sum_{x_sh} w_sh(x_sh) Omega_B(z ^ s_B(x_sh)) A_other(x_sh), and
// rounding errors of different determinants are independent, so
// Var(d amp) = (K u)^2 sum_{B,z} |C_B(z)|^2 (|det|^2 er2 + zabs2).
//
// With pattern coordinates z = (h, l), l the r_loc bits of the local gates,
// A_B(x_sh) = F_B(s_B(x_sh)) where F_B(h, m) = sum_l Omega_B(l) det_B(h, l ^ m)
// is an XOR convolution over l. When the 2^r values of both blocks fit in
// shared memory (C.wht) it is taken as a Walsh-Hadamard transform over l, a
// product with the transformed weights and the inverse transform:
// 4 r_loc 2^r real additions and 2^r complex products per block instead of
// 2^(k_sh + r_loc) complex multiply-adds.

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---- float-pair LU for the listed determinants of EF_PREC_AUTO (the FP32
// results whose error estimate called for a recompute). On this GPU an FP64
// instruction costs a warp about 64 cycles of its sub-partition's FP64 unit
// whatever its active lanes, so the thread-per-determinant FP64 LU ran as
// long as one warp's serial FP64 stream (about 40 us for the 32-qubit
// workload's 10^4 listed determinants). Float pairs (about 48 bits) run on
// the FP32 pipes. The result is stored as a float pair, as the FP64 one was.

__device__ __forceinline__ float2 ff_sub(float2 x, float2 y) { return ff_add(x, ff_neg(y)); }
// 1 / x for x > 0: the FP32 reciprocal refined by one Newton step in float
// pairs, r = r0 + r0 (1 - x r0) (as in Bailey's double-double division)
__device__ __forceinline__ float2 ff_recip(float2 x) {
    const float r0 = 1.0f / x.x;
    const float2 e = ff_sub(make_float2(1.f, 0.f), ff_mul(x, make_float2(r0, 0.f)));
    return ff_add(make_float2(r0, 0.f), ff_mul(make_float2(r0, 0.f), e));
}
__device__ __forceinline__ float4 cf_shfl(float4 v, int src, int width) {
    const unsigned full = 0xffffffffu;
    return make_float4(__shfl_sync(full, v.x, src, width), __shfl_sync(full, v.y, src, width),
                       __shfl_sync(full, v.z, src, width), __shfl_sync(full, v.w, src, width));
}

// A group of G lanes (G a power of two, eta <= G <= 32) factors one listed
// minor; lane r holds row r (float pairs) and the rows never move: at step k
// the group picks the pivot row p (largest |a_rk|^2 of the leading parts
// among rows not yet used, lowest r on ties), broadcasts its entries, and the
// other unused rows eliminate against it. The sign of the permutation is the
// parity of the unused rows below p at each step.
template <int G>
__global__ void __launch_bounds__(128) k_exact_lu_ffm(ExactBlockDev B0, ExactBlockDev B1, int nblk,
                                                      const uint64_t* __restrict__ bits,
                                                      const int2* __restrict__ mlist0,
                                                      const int2* __restrict__ mlist1,
                                                      const int* __restrict__ mcount) {
    cudaGridDependencySynchronize();  // see launch_pdl
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int r = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    constexpr int GPW = 32 / G;
    const int64_t c0 = mcount[0];
    const int64_t count = c0 + (nblk > 1 ? (int64_t)mcount[1] : 0);
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wbase = warp_global * GPW; wbase < count; wbase += nwarps * GPW) {
        const int64_t item = wbase + lane / G;
        const bool valid = item < count;
        const bool second = valid && item >= c0;
        const ExactBlockDev& B = second ? B1 : B0;
        const int eta = B.eta;
        int64_t pos = 0;
        int z = 0, row_idx = -1, cnt = -1;
        if (valid) {
            const int2 e = second ? mlist1[item - c0] : mlist0[item];
            pos = e.x;
            z = e.y;
            row_idx = nth_row(bits[2 * pos], bits[2 * pos + 1], B.mask0, B.mask1, r, cnt);
        }
        const bool ok = valid && cnt == eta;
        // the row as float pairs: leading parts from the FP32 branch matrix, the
        // rest of the FP64 value from its companion (both written by the builder)
        float4 row[G];
        const size_t src = ((size_t)z * B.n + (size_t)(row_idx < 0 ? 0 : row_idx)) * eta;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            row[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok && r < eta && j < eta) {
                const float2 h = B.M32[src + j], l = B.ML32[src + j];
                row[j] = make_float4(h.x, h.y, l.x, l.y);
            }
        }
        bool done = !ok || r >= eta;
        float4 d = make_float4(1.f, 0.f, 0.f, 0.f);
        int inv = 0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k >= eta) break;  // eta is the same in every lane of a warp (both blocks share it)
            float mag = done ? -1.f : fmaf(row[k].x, row[k].x, row[k].y * row[k].y);
            int idx = r;
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const float om = __shfl_xor_sync(full, mag, off, G);
                const int oi = __shfl_xor_sync(full, idx, off, G);
                if (om > mag || (om == mag && oi < idx)) {
                    mag = om;
                    idx = oi;
                }
            }
            const int p = idx;
            const unsigned act = (__ballot_sync(full, !done) >> gbase) & gmask;
            inv += __popc(act & ((1u << p) - 1u));
            const float4 piv = cf_shfl(row[k], p, G);
            d = cf_mul(d, piv);
            // 1 / pivot = conj(pivot) / |pivot|^2; a vanishing pivot leaves det 0 and
            // the rows unchanged
            const float2 pr = cf_re(piv), pi = cf_im(piv);
            const float2 n2 = ff_add(ff_mul(pr, pr), ff_mul(pi, pi));
            const bool nz = n2.x >= 1.17549435e-38f;
            const float2 rn = nz ? ff_recip(n2) : make_float2(0.f, 0.f);
            const float2 ipr = ff_mul(pr, rn), ipi = ff_neg(ff_mul(pi, rn));
            const bool upd = !done && r != p;
            const float4 l = cf_mul(row[k], cf_make(ipr, ipi));
#pragma unroll
            for (int j = k + 1; j < G; ++j) {
                if (j >= eta) break;
                const float4 pj = cf_shfl(row[j], p, G);
                if (upd) row[j] = cf_sub(row[j], cf_mul(l, pj));
            }
            if (r == p) done = true;
        }
        if (valid && r == 0) {
            const float4 det = !ok ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : ((inv & 1) ? make_float4(-d.x, -d.y, -d.z, -d.w) : d);
            const size_t o = dix(pos, (uint32_t)z, B.r);
            reinterpret_cast<float4*>(B.D64)[o] = det;
            B.E32[o] = kErrRedone;
        }
    }
}

cudaError_t launch_exact_lu_redo_minors(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk,
                                        const uint64_t* bits, const int2* mlist0, const int2* mlist1,
                                        const int* mcount, cudaStream_t s, LaunchStats& st) {
    if (nblk > 1 && b1.eta != b0.eta) return cudaErrorInvalidValue;
    if (b0.eta < 1 || b0.eta > 16) return cudaErrorInvalidValue;
    st.launches += 1;
    // the count lives on the device: a fixed grid of one wave strides over the list
    const int grid = sm_count() * 4;
    const int eta = b0.eta;
    cudaError_t le;
    if (eta <= 2) le = launch_pdl(k_exact_lu_ffm<2>, dim3(grid), dim3(128), 0, s, b0, b1, nblk, bits, mlist0, mlist1, mcount);
    else if (eta <= 4) le = launch_pdl(k_exact_lu_ffm<4>, dim3(grid), dim3(128), 0, s, b0, b1, nblk, bits, mlist0, mlist1, mcount);
    else if (eta <= 8) le = launch_pdl(k_exact_lu_ffm<8>, dim3(grid), dim3(128), 0, s, b0, b1, nblk, bits, mlist0, mlist1, mcount);
    else le = launch_pdl(k_exact_lu_ffm<16>, dim3(grid), dim3(128), 0, s, b0, b1, nblk, bits, mlist0, mlist1, mcount);
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

// Walsh-Hadamard stage over bit j on float pairs, optionally followed by the
// product with W[index & lm].
__device__ __forceinline__ void wht_stage_ff(float4* F, int half, int j, const float4* W, uint32_t lm, int tid,
                                             int nt) {
    for (int q = tid; q < half; q += nt) {
        const int i0 = ((q >> j) << (j + 1)) | (q & ((1 << j) - 1));
        const int i1 = i0 | (1 << j);
        const float4 a = F[i0], b = F[i1];
        float4 u = cf_add(a, b);
        float4 v = cf_sub(a, b);
        if (W) {
            u = cf_mul(u, W[i0 & lm]);
            v = cf_mul(v, W[i1 & lm]);
        }
        F[i0] = u;
        F[i1] = v;
    }
}

// float -> double by integer operations (exact; no FP64 instruction). On this
// GPU every FP64 instruction, even with one active lane or predicated off,
// holds the SM sub-partition's FP64 unit for tens of cycles, so the fast
// combines keep FP64 out of their per-bitstring code.
__device__ __forceinline__ double f2d_int(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint32_t ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
    uint64_t bits;
    if (ex == 0xffu) {
        bits = sign | 0x7ff0000000000000ull | ((uint64_t)man << 29);
    } else if (ex != 0u) {
        bits = sign | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)man << 29);
    } else if (man == 0u) {
        bits = sign;
    } else {  // subnormal float: normal in double
        const int lz = __clz(man);  // leading one at bit 31 - lz
        bits = sign | ((uint64_t)(905 - lz) << 52) | ((uint64_t)((man << (lz - 8)) & 0x7fffffu) << 29);
    }
    return __longlong_as_double((long long)bits);
}
// -|x| by setting the sign bit
__device__ __forceinline__ double neg_abs_int(double x) {
    return __longlong_as_double(__double_as_longlong(x) | (long long)0x8000000000000000ull);
}

// Determinant z of block B for D column col, as the combine's source says. A
// determinant redone for a marked FP32 entry is stored as a float pair
// (re hi, im hi, re lo, im lo) in its D64 slot.
__device__ __forceinline__ double2 det_at(const ExactCombineDev& C, int B, size_t idx) {
    if (C.src == 1) return C.D64[B][idx];
    if (C.src == 2 && err_redone(C.E32[B][idx])) {
        const float4 f = reinterpret_cast<const float4*>(C.D64[B])[idx];
        return make_double2((double)f.x + (double)f.z, (double)f.y + (double)f.w);
    }
    const float2 v = C.D32[B][idx];
    return make_double2((double)v.x, (double)v.y);
}
// the stored error term of an FP32 determinant (0 for a redone one)
__device__ __forceinline__ float err_term(const ExactCombineDev& C, int B, size_t idx) {
    return err_term_value(C.E32[B][idx]);
}

// Butterfly over lane bit j of a value held one per lane: the lane whose
// element index has bit j clear gets v + partner, the other partner - v.
__device__ __forceinline__ float4 lane_butterfly(float4 v, int j, bool upper) {
    float4 o;
    o.x = __shfl_xor_sync(0xffffffffu, v.x, 1 << j);
    o.y = __shfl_xor_sync(0xffffffffu, v.y, 1 << j);
    o.z = __shfl_xor_sync(0xffffffffu, v.z, 1 << j);
    o.w = __shfl_xor_sync(0xffffffffu, v.w, 1 << j);
    return cf_add(o, upper ? make_float4(-v.x, -v.y, -v.z, -v.w) : v);
}
__device__ __forceinline__ float2 lane_butterfly(float2 v, int j, bool upper) {
    const float ox = __shfl_xor_sync(0xffffffffu, v.x, 1 << j);
    const float oy = __shfl_xor_sync(0xffffffffu, v.y, 1 << j);
    return upper ? make_float2(ox - v.x, oy - v.y) : make_float2(v.x + ox, v.y + oy);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ float4 warp_sum_cf(float4 v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        float4 o;
        o.x = __shfl_xor_sync(0xffffffffu, v.x, off);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, off);
        o.z = __shfl_xor_sync(0xffffffffu, v.z, off);
        o.w = __shfl_xor_sync(0xffffffffu, v.w, off);
        v = cf_add(v, o);
    }
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// One stage of an in-place Walsh-Hadamard transform over bit j of F's index
// (n/2 butterflies), optionally followed by the product with W[index & lm].
__device__ __forceinline__ void wht_stage(double2* F, int half, int j, const double2* W, uint32_t lm, int tid,
                                          int nt) {
    for (int q = tid; q < half; q += nt) {
        const int i0 = ((q >> j) << (j + 1)) | (q & ((1 << j) - 1));
        const int i1 = i0 | (1 << j);
        const double2 a = F[i0], b = F[i1];
        double2 u = make_double2(a.x + b.x, a.y + b.y);
        double2 v = make_double2(a.x - b.x, a.y - b.y);
        if (W) {
            u = cmul_d(u, W[i0 & lm]);
            v = cmul_d(v, W[i1 & lm]);
        }
        F[i0] = u;
        F[i1] = v;
    }
}

__global__ void __launch_bounds__(256, 3) k_exact_combine(ExactCombineDev C, const uint64_t* __restrict__ bits,
                                                       int64_t nb, int64_t stride, const int* __restrict__ list,
                                                       const int* __restrict__ list_count, double* __restrict__ out,
                                                       double* __restrict__ err, int* __restrict__ append_list,
                                                       int* __restrict__ append_count) {
    cudaGridDependencySynchronize();  // see launch_pdl
    constexpr int NT = 256;
    constexpr int NW = NT / 32;
    // dynamic shared memory: [F_0 (2^r_0), F_1 (2^r_1), 16 bytes each, when C.wht:
    // double2, or float pairs over FP32 determinants] [FP32 copies of A_0, A_1
    // (2^k_sh each) for the error estimate] [the variance term of every
    // determinant (2^r_0 + 2^r_1 floats) when listing the ones to redo in FP64]
    extern __shared__ double2 smDyn[];
    __shared__ double red[2 * NW];
    __shared__ float4 redf[NW];
    __shared__ float redv[NW];
    __shared__ double s_theta;
    const int nsh = 1 << C.k_sh;
    const int nF = C.wht ? (1 << C.r[0]) + (1 << C.r[1]) : 0;
    const bool ffw = C.wht && C.src == 0;  // transforms on float pairs
    double2* F0 = smDyn;
    double2* F1 = smDyn + (C.wht ? (1 << C.r[0]) : 0);
    float4* G0 = reinterpret_cast<float4*>(F0);
    float4* G1 = reinterpret_cast<float4*>(F1);
    float2* smA32 = reinterpret_cast<float2*>(smDyn + nF);
    float* smV = reinterpret_cast<float*>(smA32 + 2 * nsh);
    const int tid = threadIdx.x;
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    if (C.recomp && blockIdx.x == 0 && tid == 0) {
        if (C.count_bits) atomicAdd(&C.recomp[0], (unsigned long long)count);
        if (C.count_full) atomicAdd(&C.recomp[1], (unsigned long long)count * (unsigned long long)C.minors);
        if (C.count_minors)
            for (int B = 0; B < C.nblocks; ++B) atomicAdd(&C.recomp[1], (unsigned long long)C.mcount[B]);
    }
    const bool want_err = C.err_coef > 0.0;
    const bool emit = want_err && !list && C.mlist[0] != nullptr;
    const int voff1 = C.nblocks == 2 ? (1 << C.r[0]) : 0;
    for (int64_t pos = blockIdx.x; pos < count; pos += gridDim.x) {
        const int64_t b = list ? (int64_t)list[pos] : pos;
        const int64_t col = C.col_by_index ? b : pos;  // column of D holding this bitstring's determinants
        const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
        bool ok = ((w0 & C.inactive0) == 0) && ((w1 & C.inactive1) == 0);
        for (int B = 0; B < C.nblocks; ++B)
            ok = ok && (__popcll(w0 & C.mask[B][0]) + __popcll(w1 & C.mask[B][1]) == C.eta[B]);
        if (!ok) {
            if (tid == 0) {
                out[b] = 0.0;
                if (err && !list) err[b] = 0.0;
            }
            continue;
        }
        double ar = 0.0, ai = 0.0;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);  // float-pair amplitude of the transform path
        float var = 0.f;
        if (C.nblocks == 0) {
            ar = tid == 0 ? 1.0 : 0.0;
        } else if (C.nblocks == 1) {
            // amp = sum_z Omega(z) det(z); C(z) = Omega(z)
            const int nz = 1 << C.r[0];
            for (int z = tid; z < nz; z += NT) {
                const size_t idx = dix(col, (uint32_t)z, C.r[0]);
                const double2 v = det_at(C, 0, idx);
                const double2 w = C.Omega[0][z];
                ar = fma(w.x, v.x, fma(-w.y, v.y, ar));
                ai = fma(w.x, v.y, fma(w.y, v.x, ai));
                if (want_err) {
                    const float2 w32 = C.Omega32[0][z];
                    const float vt = fmaf(w32.x, w32.x, w32.y * w32.y) * err_term(C, 0, idx);
                    var += vt;
                    if (emit) smV[z] = vt;
                }
            }
        } else if (ffw) {
            // FP32 determinants: transforms and products on float pairs
            for (int B = 0; B < 2; ++B) {
                float4* GB = B ? G1 : G0;
                const int nz = 1 << C.r[B];
                for (int z = tid; z < nz; z += NT) {
                    const float2 v = C.D32[B][dix(col, (uint32_t)z, C.r[B])];
                    GB[z] = cf_from_f(v);
                }
            }
            __syncthreads();
            const int rl = max(C.r_loc[0], C.r_loc[1]);
            for (int pass = 0; pass < 2; ++pass)
                for (int j = 0; j < rl; ++j) {
                    for (int B = 0; B < 2; ++B) {
                        if (j >= C.r_loc[B]) continue;
                        const bool mul = pass == 0 && j == C.r_loc[B] - 1;
                        wht_stage_ff(B ? G1 : G0, 1 << (C.r[B] - 1), j, mul ? C.OmegaHatDF[B] : nullptr,
                                     (1u << C.r_loc[B]) - 1u, tid, NT);
                    }
                    __syncthreads();
                }
            for (int xs = tid; xs < nsh; xs += NT) {
                const float4 a0 = G0[C.s[0][xs]], a1 = G1[C.s[1][xs]];
                if (want_err) {
                    smA32[xs] = cf_hi(a0);
                    smA32[nsh + xs] = cf_hi(a1);
                }
                acc = cf_add(acc, cf_mul(C.WSDF[xs], cf_mul(a0, a1)));
            }
        } else if (C.wht) {
            for (int B = 0; B < 2; ++B) {
                double2* FB = B ? F1 : F0;
                const int nz = 1 << C.r[B];
                for (int z = tid; z < nz; z += NT) FB[z] = det_at(C, B, dix(col, (uint32_t)z, C.r[B]));
            }
            __syncthreads();
            // forward transform (the last stage also multiplies by the transformed
            // weights, which carry the inverse's 2^-r_loc), then the inverse
            const int rl = max(C.r_loc[0], C.r_loc[1]);
            for (int pass = 0; pass < 2; ++pass)
                for (int j = 0; j < rl; ++j) {
                    for (int B = 0; B < 2; ++B) {
                        if (j >= C.r_loc[B]) continue;
                        const bool mul = pass == 0 && j == C.r_loc[B] - 1;
                        wht_stage(B ? F1 : F0, 1 << (C.r[B] - 1), j, mul ? C.OmegaHat[B] : nullptr,
                                  (1u << C.r_loc[B]) - 1u, tid, NT);
                    }
                    __syncthreads();
                }
            for (int xs = tid; xs < nsh; xs += NT) {
                const double2 a0 = F0[C.s[0][xs]], a1 = F1[C.s[1][xs]];
                if (want_err) {
                    smA32[xs] = make_float2((float)a0.x, (float)a0.y);
                    smA32[nsh + xs] = make_float2((float)a1.x, (float)a1.y);
                }
                const double2 t = cmul_d(C.WS[xs], cmul_d(a0, a1));
                ar += t.x;
                ai += t.y;
            }
        } else {
            const int nl0 = 1 << C.r_loc[0], nl1 = 1 << C.r_loc[1];
            for (int xs = tid; xs < nsh; xs += NT) {
                double2 a[2];
                for (int B = 0; B < 2; ++B) {
                    const uint32_t sB = C.s[B][xs];
                    const int nl = B == 0 ? nl0 : nl1;
                    double sx = 0.0, sy = 0.0;
                    for (int zl = 0; zl < nl; ++zl) {
                        const double2 v = det_at(C, B, dix(col, (uint32_t)zl ^ sB, C.r[B]));
                        const double2 w = C.Omega[B][zl];
                        sx = fma(w.x, v.x, fma(-w.y, v.y, sx));
                        sy = fma(w.x, v.y, fma(w.y, v.x, sy));
                    }
                    a[B] = make_double2(sx, sy);
                    if (want_err) smA32[B * nsh + xs] = make_float2((float)sx, (float)sy);
                }
                const double2 t = cmul_d(C.WS[xs], cmul_d(a[0], a[1]));
                ar += t.x;
                ai += t.y;
            }
        }
        // amplitude: warp butterflies, then thread 0 adds the warps' partial sums
        // in a fixed order
        if (ffw) {
            acc = warp_sum_cf(acc);
            if ((tid & 31) == 0) redf[tid >> 5] = acc;
        } else {
            ar = warp_sum(ar);
            ai = warp_sum(ai);
            if ((tid & 31) == 0) {
                red[tid >> 5] = ar;
                red[NW + (tid >> 5)] = ai;
            }
        }
        if (want_err && C.nblocks == 2) {
            __syncthreads();  // smA32 complete
            // the estimate needs no FP64: coefficients and terms in FP32
            for (int B = 0; B < 2; ++B) {
                const int nz = 1 << C.r[B];
                const uint32_t lmask = (1u << C.r_loc[B]) - 1u;
                const float2* Aoth = smA32 + (1 - B) * nsh;
                for (int z = tid; z < nz; z += NT) {
                    const uint32_t h = (uint32_t)z >> C.r_loc[B];
                    float cx = 0.f, cy = 0.f;
                    for (uint32_t g = C.goff[B][h]; g < C.goff[B][h + 1]; ++g) {
                        const uint32_t xs = C.perm[B][g];
                        const uint32_t zl = ((uint32_t)z ^ C.s[B][xs]) & lmask;
                        const float2 t = cmul(C.WS32[xs], cmul(C.Omega32[B][zl], Aoth[xs]));
                        cx += t.x;
                        cy += t.y;
                    }
                    const float vt = fmaf(cx, cx, cy * cy) * err_term(C, B, dix(col, (uint32_t)z, C.r[B]));
                    var += vt;
                    if (emit) smV[B * voff1 + z] = vt;
                }
            }
        }
        var = warp_sum_f(var);
        if ((tid & 31) == 0) redv[tid >> 5] = var;
        __syncthreads();
        if (tid == 0) {
            if (ffw) {
                acc = redf[0];
                for (int w = 1; w < NW; ++w) acc = cf_add(acc, redf[w]);
                ar = (double)acc.x + (double)acc.z;
                ai = (double)acc.y + (double)acc.w;
            } else {
                ar = red[0];
                ai = red[NW];
                for (int w = 1; w < NW; ++w) {
                    ar += red[w];
                    ai += red[NW + w];
                }
            }
            const double p = ar * ar + ai * ai;
            double dvar = 0.0;
            for (int w = 0; w < NW; ++w) dvar += (double)redv[w];
            // |p~ - p| <= 2 |amp| s + s^2 for an amplitude error of size s
            const double sp = sqrt(p);
            const double sig = C.err_coef * sqrt(dvar);
            const double e = fma(2.0 * sp, sig, sig * sig) / fmax(p, C.p_floor);
            out[b] = p;
            if (list) {
                if (err) err[b] = -fabs(err[b]);
            } else if (err) {
                err[b] = e;
            }
            const bool flag = append_list && e > C.tol;
            if (flag) {
                const int idx = atomicAdd(append_count, 1);
                append_list[idx] = (int)b;
            }
            if (emit) {
                // variance at which the estimate equals tol (s_t: root of
                // 2 sp s + s^2 = tol max(p, floor)); determinants whose term exceeds
                // half of it shared over all of them are redone, so the terms left
                // cannot sum past half of it
                const double st = C.tol * fmax(p, C.p_floor) / (sp + sqrt(fma(C.tol, fmax(p, C.p_floor), p)));
                const double vt = st / C.err_coef;
                s_theta = flag ? 0.5 * vt * vt / (double)C.minors : -1.0;
            }
        }
        if (emit) {
            __syncthreads();
            const double theta = s_theta;
            if (theta >= 0.0)
                for (int B = 0; B < C.nblocks; ++B) {
                    const int nz = 1 << C.r[B];
                    for (int z = tid; z < nz; z += NT)
                        if ((double)smV[B * voff1 + z] > theta) {
                            const int idx = atomicAdd(&C.mcount[B], 1);
                            C.mlist[B][idx] = make_int2((int)pos, z);
                        }
                }
        }
        __syncthreads();
    }
}

// Primary pass over FP32 determinants when both blocks have 32 <= 2^r <= 1024
// patterns and at most 5 local pattern bits (ExactCombineDev.wreg). Same
// arithmetic as k_exact_combine's float-pair path, organised for throughput:
//  * thread <-> elements e = tid + NT i of each block, so the local pattern
//    bits are lane bits and both transforms (float pairs for the amplitude,
//    FP32 for the error coefficients) run in registers by shuffles;
//  * the error coefficients are XOR convolutions too: C_B(h, .) = Omega_B
//    convolved with Q_B(h, .), Q_B(z) = sum of w_sh A_other over the x_sh with
//    s_B(x_sh) = z;
//  * shared memory is double-buffered by iteration parity and each
//    bitstring's totals, flag and determinant list are finished by one warp
//    (rotating), so no CTA-wide barrier waits for that serial tail.
template <int NT>
__global__ void __launch_bounds__(NT, 3) k_exact_combine_ffr(ExactCombineDev C, const uint64_t* __restrict__ bits,
                                                             int64_t nb, int64_t stride, const int* __restrict__ list,
                                                             const int* __restrict__ list_count,
                                                             double* __restrict__ out, double* __restrict__ err,
                                                             int* __restrict__ append_list,
                                                             int* __restrict__ append_count) {
    cudaGridDependencySynchronize();  // see launch_pdl
    constexpr int NW = NT / 32;
    extern __shared__ float4 smF[];
    __shared__ float4 redf[2][NW];
    __shared__ float redv[2][NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsh = 1 << C.k_sh;
    const int n0 = 1 << C.r[0], n1 = 1 << C.r[1];
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    if (C.recomp && blockIdx.x == 0 && tid == 0) {
        if (C.count_bits) atomicAdd(&C.recomp[0], (unsigned long long)count);
        if (C.count_minors)
            for (int B = 0; B < 2; ++B) atomicAdd(&C.recomp[1], (unsigned long long)C.mcount[B]);
    }
    const bool want_err = C.err_coef > 0.0;
    const bool emit = want_err && !list && C.mlist[0] != nullptr;
    const float floor_f = (float)C.p_floor, tol_f = (float)C.tol, ec_f = (float)C.err_coef;
    // per buffer: G_0 (n0), G_1 (n1) float4; A_0, A_1 (nsh each) float2; V (n0 + n1) float
    const size_t buf_words = (size_t)4 * (n0 + n1) + (size_t)4 * nsh + (emit ? (size_t)(n0 + n1) : 0);
    int it = 0;
    for (int64_t pos = blockIdx.x; pos < count; pos += gridDim.x, ++it) {
        const int64_t b = list ? (int64_t)list[pos] : pos;
        const int64_t col = C.col_by_index ? b : pos;  // column of D holding this bitstring's determinants
        const int buf = it & 1;
        float* base = reinterpret_cast<float*>(smF) + (size_t)buf * buf_words;
        float4* G0 = reinterpret_cast<float4*>(base);
        float4* G1 = G0 + n0;
        float2* A32 = reinterpret_cast<float2*>(G1 + n1);
        float* V = reinterpret_cast<float*>(A32 + 2 * nsh);
        const int tail = it % NW;  // warp that finishes this bitstring
        const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
        bool ok = ((w0 & C.inactive0) == 0) && ((w1 & C.inactive1) == 0);
        for (int B = 0; B < 2; ++B)
            ok = ok && (__popcll(w0 & C.mask[B][0]) + __popcll(w1 & C.mask[B][1]) == C.eta[B]);
        if (!ok) {
            if (tid == 0) {
                out[b] = 0.0;
                if (err && !list) err[b] = 0.0;
            }
            continue;
        }
        float errt[2][kWregMax];
        // 1. F_B = Omega_B convolved with det_B over the local bits (float pairs)
#pragma unroll
        for (int B = 0; B < 2; ++B) {
            const int nz = B ? n1 : n0;
            const int rl = C.r_loc[B];
            const uint32_t lm = (1u << rl) - 1u;
            float4* GB = B ? G1 : G0;
#pragma unroll
            for (int i = 0; i < kWregMax; ++i) {
                const int e = tid + NT * i;
                if (e >= nz) break;
                const size_t idx = dix(col, (uint32_t)e, C.r[B]);
                const float2 d = C.D32[B][idx];
                const uint16_t ec = C.E32[B][idx];
                errt[B][i] = want_err ? err_term_value(ec) : 0.f;
                float4 v = cf_from_f(d);
                if (C.src == 2 && err_redone(ec))  // redone, stored as a float pair
                    v = reinterpret_cast<const float4*>(C.D64[B])[idx];
                for (int pass = 0; pass < 2; ++pass)
                    for (int j = 0; j < rl; ++j) {
                        v = lane_butterfly(v, j, (e >> j) & 1);
                        if (pass == 0 && j == rl - 1) v = cf_mul(v, C.OmegaHatDF[B][e & lm]);
                    }
                GB[e] = v;
            }
        }
        __syncthreads();
        // 2. amp = sum_xs WS(xs) F_0(s_0(xs)) F_1(s_1(xs))
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int xs = tid; xs < nsh; xs += NT) {
            const float4 a0 = G0[C.s[0][xs]], a1 = G1[C.s[1][xs]];
            A32[xs] = cf_hi(a0);
            A32[nsh + xs] = cf_hi(a1);
            acc = cf_add(acc, cf_mul(C.WSDF[xs], cf_mul(a0, a1)));
        }
        float var = 0.f;
        if (want_err) {
            __syncthreads();  // A32 complete
#pragma unroll
            for (int B = 0; B < 2; ++B) {
                const int nz = B ? n1 : n0;
                const int rl = C.r_loc[B];
                const uint32_t lm = (1u << rl) - 1u;
                const float2* Aoth = A32 + (1 - B) * nsh;
#pragma unroll
                for (int i = 0; i < kWregMax; ++i) {
                    const int e = tid + NT * i;
                    if (e >= nz) break;
                    float2 q = make_float2(0.f, 0.f);
                    for (uint32_t g = C.inv_off[B][e]; g < C.inv_off[B][e + 1]; ++g) {
                        const uint32_t xs = C.inv_xs[B][g];
                        const float2 t = cmul(C.WS32[xs], Aoth[xs]);
                        q.x += t.x;
                        q.y += t.y;
                    }
                    for (int pass = 0; pass < 2; ++pass)
                        for (int j = 0; j < rl; ++j) {
                            q = lane_butterfly(q, j, (e >> j) & 1);
                            if (pass == 0 && j == rl - 1) {
                                const float4 w = C.OmegaHatDF[B][e & lm];
                                q = pcmul(q, cf_hi(w));
                            }
                        }
                    const float vt = fmaf(q.x, q.x, q.y * q.y) * errt[B][i];
                    var += vt;
                    if (emit) V[B * n0 + e] = vt;
                }
            }
        }
        acc = warp_sum_cf(acc);
        var = warp_sum_f(var);
        if (lane == 0) {
            redf[buf][warp] = acc;
            redv[buf][warp] = var;
        }
        __syncthreads();
        if (warp != tail) continue;
        // 3. the tail warp: totals in a fixed order (lanes 0..NW-1 then butterflies)
        float4 a = lane < NW ? redf[buf][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        float vv = lane < NW ? redv[buf][lane] : 0.f;
#pragma unroll
        for (int off = NW / 2; off > 0; off >>= 1) {
            float4 o;
            o.x = __shfl_xor_sync(0xffffffffu, a.x, off);
            o.y = __shfl_xor_sync(0xffffffffu, a.y, off);
            o.z = __shfl_xor_sync(0xffffffffu, a.z, off);
            o.w = __shfl_xor_sync(0xffffffffu, a.w, off);
            a = cf_add(a, o);
            vv += __shfl_xor_sync(0xffffffffu, vv, off);
        }
        float budget = -1.f;
        if (lane == 0) {
            // p = |amp|^2 in float pairs; one FP64 addition forms the output
            const float2 pff = ff_add(ff_mul(cf_re(a), cf_re(a)), ff_mul(cf_im(a), cf_im(a)));
            out[b] = f2d_int(pff.x) + f2d_int(pff.y);
            // error estimate in FP32: |p~ - p| <= 2 |amp| s + s^2 for an amplitude error s
            const float pf = pff.x, tol = tol_f, ec = ec_f;
            const float pm = fmaxf(pf, floor_f);
            const float sp = sqrtf(pf);
            const float sig = ec * sqrtf(vv);
            const float e = want_err ? fmaf(2.f * sp, sig, sig * sig) / pm : 0.f;
            if (list) {
                if (err) err[b] = neg_abs_int(err[b]);
            } else if (err) {
                err[b] = f2d_int(e);
            }
            if (append_list && !(e <= tol)) {
                append_list[atomicAdd(append_count, 1)] = (int)b;
                if (emit) {
                    // half the variance at which the estimate equals tol
                    const float st = tol * pm / (sp + sqrtf(fmaf(tol, pm, pf)));
                    const float vt = st / ec;
                    budget = 0.5f * vt * vt;
                }
            }
        }
        budget = __shfl_sync(0xffffffffu, budget, 0);
        if (budget >= 0.f) {
            // the largest threshold t whose terms <= t sum to at most the budget
            // (bisection on the bit patterns of non-negative floats); the
            // determinants with larger terms are redone in float pairs
            uint32_t lo = 0u, hi = 0x7f800000u;  // [0, +inf]
            while (hi - lo > 1u) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                const float t = __uint_as_float(mid);
                float sum = 0.f;
                for (int z = lane; z < n0 + n1; z += 32) {
                    const float v = V[z];
                    sum += v <= t ? v : 0.f;
                }
                sum = warp_sum_f(sum);
                if (sum <= budget) lo = mid;
                else hi = mid;
            }
            const float t = __uint_as_float(lo);
            for (int B = 0; B < 2; ++B) {
                const int nz = B ? n1 : n0;
                for (int z = lane; z < nz; z += 32)
                    if (!(V[B * n0 + z] <= t)) C.mlist[B][atomicAdd(&C.mcount[B], 1)] = make_int2((int)pos, z);
            }
        }
    }
}

// In-register Walsh-Hadamard transform of NL = 2^RL values (one row of a block).
template <int RL, typename T, typename Add, typename Sub>
__device__ __forceinline__ void row_wht(T (&v)[1 << RL], Add add, Sub sub) {
#pragma unroll
    for (int j = 0; j < RL; ++j)
#pragma unroll
        for (int l = 0; l < (1 << RL); ++l)
            if (!(l & (1 << j))) {
                const T a = v[l], c = v[l | (1 << j)];
                v[l] = add(a, c);
                v[l | (1 << j)] = sub(a, c);
            }
}

// Warp per bitstring: the primary and re-estimating passes over FP32
// determinants when both blocks have RL local pattern bits. A pattern
// z = (h, l) belongs to row (B, h); a lane owns whole rows, so the XOR
// convolutions over l (float pairs for the amplitude, FP32 for the error
// coefficients) run inside one thread, and a warp never waits for another.
// The arithmetic is that of k_exact_combine's float-pair path; the warp's
// shared memory holds F_B (float pairs), then A_B (FP32) and the variance
// terms for the determinant list.
template <int RL, int RPL>
__global__ void __launch_bounds__(128, (RL >= 5 ? 2 : 3)) k_exact_combine_wp(ExactCombineDev C, const uint64_t* __restrict__ bits,
                                                          int64_t nb, int64_t stride, const int* __restrict__ list,
                                                          const int* __restrict__ list_count,
                                                          double* __restrict__ out, double* __restrict__ err,
                                                          int* __restrict__ append_list,
                                                          int* __restrict__ append_count) {
    cudaGridDependencySynchronize();  // see launch_pdl
    constexpr int NL = 1 << RL;  // RPL: rows per lane at most
    extern __shared__ float4 smWp[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n0 = 1 << C.r[0], n1 = 1 << C.r[1];
    const int rows0 = n0 >> RL, rows = rows0 + (n1 >> RL);
    const int nsh = 1 << C.k_sh;
    const int64_t count = list ? (int64_t)(*list_count) : nb;
    if (C.recomp && blockIdx.x == 0 && threadIdx.x == 0) {
        if (C.count_bits) atomicAdd(&C.recomp[0], (unsigned long long)count);
        if (C.count_minors)
            for (int B = 0; B < 2; ++B) atomicAdd(&C.recomp[1], (unsigned long long)C.mcount[B]);
    }
    const bool want_err = C.err_coef > 0.0;
    const bool emit = want_err && !list && C.mlist[0] != nullptr;
    const float floor_f = (float)C.p_floor, tol_f = (float)C.tol, ec_f = (float)C.err_coef;
    // per warp: G_0, G_1 (n0 + n1 float4; after step 2 reused for V, n0 + n1
    // float) | A_0, A_1 (2 nsh float2) or, when every s_B is one-to-one (C.inj),
    // Q_0, Q_1 (n0 + n1 float2) scattered in step 2
    const size_t warp_f4 = (size_t)(n0 + n1) + (size_t)max(nsh, (n0 + n1 + 1) / 2);
    float4* G = smWp + (size_t)wib * warp_f4;
    float2* A32 = reinterpret_cast<float2*>(G + n0 + n1);
    float2* Q = A32;
    float* V = reinterpret_cast<float*>(G);
    // G, Q and V hold pattern z = (h, l) of block B at offset (B ? n0 : 0) +
    // (l << sh_B) + h (h the row, l the local bits): the NL values of a lane's
    // row then lie rows apart, and a warp's accesses to one l are consecutive
    // (with z as the index they were 2^RL apart: 32-way bank conflicts).
    // (C.r[B] - RL read from the parameter space where needed: two more live
    // registers made the kernel spill)
    const auto phys = [&](int B, uint32_t z) -> int {
        return (int)(((z & (uint32_t)(NL - 1)) << (C.r[B] - RL)) | (z >> RL));
    };
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t pos = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; pos < count; pos += nwarps) {
        const int64_t b = list ? (int64_t)list[pos] : pos;
        const int64_t col = C.col_by_index ? b : pos;
        const uint64_t w0 = bits[2 * b], w1 = bits[2 * b + 1];
        bool ok = ((w0 & C.inactive0) == 0) && ((w1 & C.inactive1) == 0);
        for (int B = 0; B < 2; ++B)
            ok = ok && (__popcll(w0 & C.mask[B][0]) + __popcll(w1 & C.mask[B][1]) == C.eta[B]);
        if (!ok) {
            if (lane == 0) {
                out[b] = 0.0;
                if (err && !list) err[b] = 0.0;
            }
            continue;
        }
        float errt[RPL][NL];
        // 1. rows of F_B = Omega_B convolved with det_B over l, in float pairs
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            const int row = lane + 32 * rr;
            if (row >= rows) break;
            const int B = row < rows0 ? 0 : 1;
            const int z0 = (B ? row - rows0 : row) << RL;
            float4 v[NL];
            // the row's NL determinants and error terms are contiguous and start at a
            // multiple of NL: read them as 16-byte (and, below 8 error terms, 4- or
            // 8-byte) vectors
            const size_t base = dix(col, (uint32_t)z0, C.r[B]);
            const float4* dv = reinterpret_cast<const float4*>(C.D32[B] + base);
            uint32_t ew[(NL + 1) / 2];
            if constexpr (NL >= 8) {
#pragma unroll
                for (int q = 0; q < NL / 8; ++q) {
                    const uint4 w = reinterpret_cast<const uint4*>(C.E32[B] + base)[q];
                    ew[4 * q] = w.x, ew[4 * q + 1] = w.y, ew[4 * q + 2] = w.z, ew[4 * q + 3] = w.w;
                }
            } else if constexpr (NL == 4) {
                const uint2 w = *reinterpret_cast<const uint2*>(C.E32[B] + base);
                ew[0] = w.x, ew[1] = w.y;
            } else {
                ew[0] = *reinterpret_cast<const uint32_t*>(C.E32[B] + base);
            }
#pragma unroll
            for (int l = 0; l < NL; l += 2) {
                const float4 dd = dv[l / 2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint16_t ec = (uint16_t)(ew[l / 2] >> (16 * h));
                    errt[rr][l + h] = want_err ? err_term_value(ec) : 0.f;
                    v[l + h] = h ? make_float4(dd.z, dd.w, 0.f, 0.f) : make_float4(dd.x, dd.y, 0.f, 0.f);
                    if (C.src == 2 && err_redone(ec))  // redone, stored as a float pair
                        v[l + h] = reinterpret_cast<const float4*>(C.D64[B])[base + l + h];
                }
            }
            row_wht<RL>(v, cf_add, cf_sub);
            const float4* Wh = C.OmegaHatDF[B];
#pragma unroll
            for (int l = 0; l < NL; ++l) v[l] = cf_mul(v[l], Wh[l]);
            row_wht<RL>(v, cf_add, cf_sub);
            float4* GB = G + (B ? n0 : 0) + (B ? row - rows0 : row);
            const int shB = C.r[B] - RL;
#pragma unroll
            for (int l = 0; l < NL; ++l) GB[l << shB] = v[l];
        }
        __syncwarp();
        // 2. amp = sum_xs WS(xs) F_0(s_0(xs)) F_1(s_1(xs)); with one-to-one s_B,
        //    also Q_B(s_B(xs)) = w_sh(xs) A_other(xs) (FP32)
        const bool scatter = want_err && C.inj;
        if (scatter) {
            for (int z = lane; z < n0 + n1; z += 32) Q[z] = make_float2(0.f, 0.f);
            __syncwarp();
        }
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int xs = lane; xs < nsh; xs += 32) {
            const int p0 = phys(0, C.s[0][xs]), p1 = n0 + phys(1, C.s[1][xs]);
            const float4 a0 = G[p0], a1 = G[p1];
            const float4 w = C.WSDF[xs];
            if (scatter) {
                const float2 w32 = cf_hi(w);
                Q[p0] = pcmul(w32, cf_hi(a1));
                Q[p1] = pcmul(w32, cf_hi(a0));
            } else if (want_err) {
                A32[xs] = cf_hi(a0);
                A32[nsh + xs] = cf_hi(a1);
            }
            acc = cf_add(acc, cf_mul(w, cf_mul(a0, a1)));
        }
        float var = 0.f;
        if (want_err) {
            __syncwarp();
            // 3. rows of C_B = Omega_B convolved with Q_B, Q_B(z) = sum of w_sh A_other
            //    over the x_sh with s_B(x_sh) = z (FP32)
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr) {
                const int row = lane + 32 * rr;
                if (row >= rows) break;
                const int B = row < rows0 ? 0 : 1;
                const int z0 = (B ? row - rows0 : row) << RL;
                // this row's entries in Q and V: NL values 1 << sh_B apart
                const int pb = (B ? n0 : 0) + (B ? row - rows0 : row), shB = C.r[B] - RL;
                const float2* Aoth = A32 + (1 - B) * nsh;
                float2 q[NL];
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    q[l] = make_float2(0.f, 0.f);
                    if (scatter) {
                        q[l] = Q[pb + (l << shB)];
                        continue;
                    }
                    for (uint32_t g = C.inv_off[B][z0 | l]; g < C.inv_off[B][(z0 | l) + 1]; ++g) {
                        const uint32_t xs = C.inv_xs[B][g];
                        q[l] = p2_add(q[l], pcmul(C.WS32[xs], Aoth[xs]));
                    }
                }
                const auto fadd = [](float2 a, float2 c) { return p2_add(a, c); };
                const auto fsub = [](float2 a, float2 c) { return p2_sub(a, c); };
                row_wht<RL>(q, fadd, fsub);
                const float4* Wh = C.OmegaHatDF[B];
#pragma unroll
                for (int l = 0; l < NL; ++l) q[l] = pcmul(q[l], cf_hi(Wh[l]));
                row_wht<RL>(q, fadd, fsub);
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const float vt = fmaf(q[l].x, q[l].x, q[l].y * q[l].y) * errt[rr][l];
                    var += vt;
                    if (emit) V[pb + (l << shB)] = vt;
                }
            }
        }
        // 4. totals (fixed butterfly order), estimate, flag, determinant list
        acc = warp_sum_cf(acc);
        var = warp_sum_f(var);
        float budget = -1.f;
        if (lane == 0) {
            // p = |amp|^2 in float pairs; one FP64 addition forms the output
            const float2 pff = ff_add(ff_mul(cf_re(acc), cf_re(acc)), ff_mul(cf_im(acc), cf_im(acc)));
            out[b] = f2d_int(pff.x) + f2d_int(pff.y);
            // |p~ - p| <= 2 |amp| s + s^2 for an amplitude error s (in FP32)
            const float pf = pff.x, tol = tol_f, ec = ec_f;
            const float pm = fmaxf(pf, floor_f);
            const float sp = sqrtf(pf);
            const float sig = ec * sqrtf(var);
            const float e = want_err ? fmaf(2.f * sp, sig, sig * sig) / pm : 0.f;
            if (list) {
                if (err) err[b] = neg_abs_int(err[b]);
            } else if (err) {
                err[b] = f2d_int(e);
            }
            if (append_list && !(e <= tol)) {
                append_list[atomicAdd(append_count, 1)] = (int)b;
                if (emit) {
                    const float st = tol * pm / (sp + sqrtf(fmaf(tol, pm, pf)));
                    const float vt = st / ec;
                    budget = 0.5f * vt * vt;  // half the variance at which the estimate equals tol
                }
            }
        }
        budget = __shfl_sync(0xffffffffu, budget, 0);
        if (budget >= 0.f) {
            __syncwarp();
            // the largest threshold whose terms sum to at most the budget, by
            // bisection on float bit patterns; larger terms are redone in float pairs
            uint32_t lo = 0u, hi = 0x7f800000u;
            while (hi - lo > 1u) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                const float t = __uint_as_float(mid);
                float sum = 0.f;
                for (int z = lane; z < n0 + n1; z += 32) {
                    const float x = V[z];
                    sum += x <= t ? x : 0.f;
                }
                if (warp_sum_f(sum) <= budget) lo = mid;
                else hi = mid;
            }
            const float t = __uint_as_float(lo);
            for (int p = lane; p < n0 + n1; p += 32)
                if (!(V[p] <= t)) {
                    const int B = p < n0 ? 0 : 1;
                    const int pz = B ? p - n0 : p, shB = C.r[B] - RL;
                    const int z = ((pz & ((1 << shB) - 1)) << RL) | (pz >> shB);  // back to (h, l)
                    C.mlist[B][atomicAdd(&C.mcount[B], 1)] = make_int2((int)pos, z);
                }
        }
        __syncwarp();
    }
}

// Shared memory per warp of k_exact_combine_wp (bytes), 0 if it does not apply.
size_t exact_combine_wp_bytes(const ExactCombineDev& c) {
    if (c.nblocks != 2 || c.r_loc[0] != c.r_loc[1] || c.r_loc[0] < 1 || c.r_loc[0] > 5) return 0;
    const int rows = (1 << (c.r[0] - c.r_loc[0])) + (1 << (c.r[1] - c.r_loc[1]));
    if (rows > 64) return 0;
    const size_t n = ((size_t)1 << c.r[0]) + ((size_t)1 << c.r[1]);
    // matches the kernel's per-warp layout
    const size_t bytes = 16 * (n + std::max(((size_t)1 << c.k_sh), (n + 1) / 2));
    return bytes <= 24 * 1024 ? bytes : 0;
}

template <int RL, int RPL>
static cudaError_t launch_wp_r(const ExactCombineDev& c, size_t per_warp, const uint64_t* bits, int64_t nb,
                               int64_t stride, const int* list, const int* list_count, double* out, double* err,
                               int* append_list, int* append_count, cudaStream_t s) {
    const size_t smem = 4 * per_warp;
    cudaError_t e = raise_dynamic_smem((const void*)k_exact_combine_wp<RL, RPL>, smem);
    if (e != cudaSuccess) return e;
    // two full waves at 3 CTAs per SM (measured: 0.563 against 0.567 ms per 32-qubit step with 8
    // CTAs per SM of grid, 2.7 waves; one wave, 0.567 ms)
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((nb + 3) / 4, (int64_t)sm_count() * 6));
    e = launch_pdl(k_exact_combine_wp<RL, RPL>, dim3((unsigned)blocks), dim3(128), smem, s, c, bits, nb, stride, list,
                   list_count, out, err, append_list, append_count);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int RL>
static cudaError_t launch_wp(const ExactCombineDev& c, size_t per_warp, const uint64_t* bits, int64_t nb,
                             int64_t stride, const int* list, const int* list_count, double* out, double* err,
                             int* append_list, int* append_count, cudaStream_t s) {
    const int rows = (1 << (c.r[0] - RL)) + (1 << (c.r[1] - RL));
    return rows <= 32 ? launch_wp_r<RL, 1>(c, per_warp, bits, nb, stride, list, list_count, out, err, append_list,
                                           append_count, s)
                      : launch_wp_r<RL, 2>(c, per_warp, bits, nb, stride, list, list_count, out, err, append_list,
                                           append_count, s);
}

size_t exact_combine_smem(const ExactCombineDev& c) {
    size_t smem = (size_t)2 * ((size_t)1 << c.k_sh) * sizeof(float2);
    if (c.wht) smem += (((size_t)1 << c.r[0]) + ((size_t)1 << c.r[1])) * sizeof(double2);
    if (c.mlist[0]) smem += (size_t)c.minors * sizeof(float);
    return smem;
}

cudaError_t launch_exact_combine(const ExactCombineDev& c, const uint64_t* bits, int64_t nb, int64_t stride,
                                 const int* list, const int* list_count, double* out, double* err, int* append_list,
                                 int* append_count, cudaStream_t s, LaunchStats& st) {
    if (nb <= 0) return cudaSuccess;
    const size_t wp = (c.src == 0 || c.src == 2) && !c.count_full ? exact_combine_wp_bytes(c) : 0;
    if (wp) {
        cudaError_t e;
        switch (c.r_loc[0]) {
            case 1: e = launch_wp<1>(c, wp, bits, nb, stride, list, list_count, out, err, append_list, append_count, s); break;
            case 2: e = launch_wp<2>(c, wp, bits, nb, stride, list, list_count, out, err, append_list, append_count, s); break;
            case 3: e = launch_wp<3>(c, wp, bits, nb, stride, list, list_count, out, err, append_list, append_count, s); break;
            case 4: e = launch_wp<4>(c, wp, bits, nb, stride, list, list_count, out, err, append_list, append_count, s); break;
            default: e = launch_wp<5>(c, wp, bits, nb, stride, list, list_count, out, err, append_list, append_count, s); break;
        }
        st.launches += 1;
        return e;
    }
    if (c.wreg && (c.src == 0 || c.src == 2) && !c.count_full) {
        constexpr int NT = 256;
        const size_t words = (size_t)4 * (((size_t)1 << c.r[0]) + ((size_t)1 << c.r[1])) +
                             (size_t)4 * ((size_t)1 << c.k_sh) +
                             (c.mlist[0] ? ((size_t)1 << c.r[0]) + ((size_t)1 << c.r[1]) : 0);
        const size_t smem = 2 * words * sizeof(float);
        cudaError_t e = raise_dynamic_smem((const void*)k_exact_combine_ffr<NT>, smem);
        if (e != cudaSuccess) return e;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)sm_count() * 12));
        e = launch_pdl(k_exact_combine_ffr<NT>, dim3((unsigned)blocks), dim3(NT), smem, s, c, bits, nb, stride, list,
                       list_count, out, err, append_list, append_count);
        if (e != cudaSuccess) return e;
        st.launches += 1;
        return cudaGetLastError();
    }
    const size_t smem = exact_combine_smem(c);
    cudaError_t e = raise_dynamic_smem((const void*)k_exact_combine, smem);
    if (e != cudaSuccess) return e;
    // a list (the FP64 pass over the results still above tol) is usually short or empty
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)sm_count() * (list ? 4 : 16)));
    e = launch_pdl(k_exact_combine, dim3((unsigned)blocks), dim3(256), smem, s, c, bits, nb, stride, list, list_count,
                   out, err, append_list, append_count);
    if (e != cudaSuccess) return e;
    st.launches += 1;
    return cudaGetLastError();
}

}  // namespace ef
