// Internal structures shared by the host runtime (ef_api.cu) and the kernels
// (ef_exact.cu, ef_approx.cu). Plain device pointers and sizes only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ef {

// One partial branch sum of the Exact path: (re, im) of sum_y w(y) det, and
// S = sum_y |w|^2 |det|^2, E = sum_y |w|^2 e_det^2 for the FP32 error estimate
struct __align__(32) d4 {
    double x, y, z, w;
};
__host__ __device__ inline d4 make_d4(double x, double y, double z, double w) { return d4{x, y, z, w}; }

constexpr int kMaxModes = 128;
constexpr int kMaxBlocks = 2;      // independent mode blocks kept factorised
constexpr int kMaxEtaRows = 32;    // warp-row LU: one lane per minor row
constexpr int kMaxEtaThread = 10;  // FP32 thread-per-minor LU (registers)
constexpr int kMaxApproxEta = 8;   // Raw Estimate, thread per trajectory
constexpr int kMaxApproxLayers = 8;
constexpr int kMaxApproxStored = 64;  // rank-one columns kept per trajectory
constexpr int kMaxExactSubBits = 24;  // 2^24 sub-branches per block

// ---------------------------------------------------------------- Exact mode

// One independent mode block of the Exact path. Sub-branch y of the block
// holds the bits of the controlled-phase gates that touch it: bits
// [0, k_loc) for gates local to the block, [k_loc, k_loc + k_sh) for gates
// shared with the other block.
struct ExactBlockDev {
    int n, eta, L;          // modes, particles, diagonal layers in this block
    int k_loc, k_sh;        // sub-branch bits
    int c_log2;             // FP32 kernel: log2 sub-branches per chunk
    int lobits;             // weight table split of the local bits
    uint64_t mask0, mask1;  // global modes of the block
    const double2* S0C;     // n x eta: first segment restricted to the occupied columns
    const double2* T;       // L x n x n: T_l = S_l diag(base phases of layer l)
    const uint32_t* F;      // L x n: flip masks over y bits, per layer and local mode
    const double* WLlo;     // 2^lobits
    const double* WLhi;     // 2^(k_loc - lobits)
    double2* M64;           // 2^(k_loc+k_sh) x n x eta branch matrices (FP64)
    float2* M32;            // same, FP32 (may be null)
    d4* part;               // [n_chunks][count]: (re, im, S, E) per chunk
    int n_chunks;           // 2^(k_loc + k_sh - c_log2)
};

struct ExactCombineDev {
    int nblocks;
    int k_sh;
    int shlobits;
    const double* WSlo;
    const double* WShi;
    uint64_t inactive0, inactive1;  // modes outside every active block (must be empty)
    uint64_t mask[kMaxBlocks][2];
    int eta[kMaxBlocks];
    int c_log2[kMaxBlocks];
    int k_loc[kMaxBlocks];
    const d4* part[kMaxBlocks];
    int eta_max;
    double err_coef;  // K * eta_max * u32 (FP32 path), 0 for FP64
    double tol, p_floor;
};

// ---------------------------------------------------------------- Raw Estimate

struct ApproxBlockDev {
    int n, eta, L;
    uint64_t mask0, mask1;
    const void* P;    // interval products Pi_{a..b}, a >= b, tri index a(a+1)/2 + b, n x n each
    const void* RC;   // L x n x eta: Pi_{l..0}[:, C] for l = 0..L-1
    const int* cols;  // eta local column indices
};

struct ApproxDev {
    int nblocks;
    int k;
    const uint32_t* T;       // thresholds
    const double* qratio;    // (s/pT1) / (c/pT0) per gate
    const uint8_t* glayer;   // [kMaxBlocks][k]: layer 1..L in the block, 0 = not touching
    const uint64_t* gmodes;  // [kMaxBlocks][k]: local modes flipped in the block
    double R0;               // prod_j c_j / pT0_j
    uint32_t key0, key1;
    uint64_t index_base;
    uint64_t inactive0, inactive1;
    int64_t t;
    int traj_per_cta;
    int n_chunks;
    double* part;                 // [nb][n_chunks][8]
    unsigned long long* counters; // [0] flips, [1] executed LUs
    ApproxBlockDev blk[kMaxBlocks];
};

// ---------------------------------------------------------------- launchers

struct LaunchStats {
    int64_t launches = 0;
    int64_t executed_lus = 0;
};

cudaError_t launch_build_branches(const ExactBlockDev& b, bool want32, cudaStream_t s, LaunchStats& st);
cudaError_t launch_exact_lu_f32(const ExactBlockDev& b, const uint64_t* bits, int64_t nb,
                                cudaStream_t s, LaunchStats& st);
cudaError_t launch_exact_lu_rows(const ExactBlockDev& b, const uint64_t* bits, int64_t nb,
                                 const int* list, const int* list_count, int64_t cap,
                                 bool fp64, cudaStream_t s, LaunchStats& st);
cudaError_t launch_exact_combine(const ExactCombineDev& c, const uint64_t* bits, int64_t nb,
                                 const int* list, const int* list_count, double* out, double* err,
                                 int* append_list, int* append_count, cudaStream_t s, LaunchStats& st);
cudaError_t launch_approx(const ApproxDev& a, const uint64_t* bits, int64_t nb, bool fp64,
                          cudaStream_t s, LaunchStats& st);
cudaError_t launch_approx_finalize(const ApproxDev& a, int64_t nb, double* out, double* stderr_out,
                                   cudaStream_t s, LaunchStats& st);

}  // namespace ef
