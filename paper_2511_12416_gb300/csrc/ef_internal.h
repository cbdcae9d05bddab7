// Internal structures shared by the host runtime (ef_api.cu) and the kernels
// (ef_exact.cu, ef_approx.cu). Plain device pointers and sizes only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ef {

constexpr int kMaxModes = 128;
constexpr int kMaxBlocks = 2;      // independent mode blocks kept factorised
constexpr int kMaxEtaRows = 32;    // warp-row LU: one lane per minor row
constexpr int kMaxEtaThread = 10;  // FP32 thread-per-minor LU (registers)
constexpr int kMaxApproxEta = 13;    // Raw Estimate, thread per trajectory, FP32 minors
constexpr int kMaxApproxEta64 = 13;  // FP64 minors
constexpr int kApproxPartStride = 11; // Raw Estimate partial sums per (bitstring, trajectory chunk)
constexpr int kMaxApproxLayers = 8;
constexpr int kMaxApproxStored = 64;  // rank-one columns kept per trajectory
constexpr int kMaxExactPatternBits = 22;  // 2^22 flip patterns per block
constexpr int kMaxExactLocalBits = 22;    // local gates per block
constexpr int kMaxExactSharedBits = 12;   // gates shared by the two blocks
constexpr int kWregMax = 4;               // elements per thread and block of the combine's register path

// ---------------------------------------------------------------- Exact mode

// One independent mode block of the Exact path. A trajectory's minor in the
// block depends on the controlled-phase bits only through its flip pattern
// (which local modes change sign in which layer), a GF(2)-linear function of
// the bits. The r basis patterns span every pattern that occurs; pattern z
// (r bits, coordinates in that basis) flips mode i of layer l iff
// popcount(z & F[l*n + i]) is odd. The first r_loc basis patterns span the
// patterns of the block's local gates.
struct ExactBlockDev {
    int n, eta, L;          // modes, particles, diagonal layers in this block
    int r, r_loc;           // pattern rank, rank of the local gates' patterns
    int c_log2;             // patterns per chunk of the FP32 kernel (log2)
    int n_chunks;           // 2^(r - c_log2)
    uint64_t mask0, mask1;  // global modes of the block
    const double2* S0C;     // n x eta: first segment restricted to the occupied columns
    const double2* T;       // L x n x n: T_l = S_l diag(base phases of layer l)
    const uint32_t* F;      // L x n: flip masks over pattern bits
    double2* M64;           // 2^r x n x eta branch matrices (FP64)
    float2* M32;            // same, FP32 (may be null)
    float2* ML32;           // with M32: M64 - M32 rounded to FP32 (M32 + ML32 = M64 to about 48 bits)
    // determinants per (bitstring column, pattern), [stride][2^r] each (dix):
    float2* D32;            // FP32 LU: det
    uint16_t* E32;          // FP32 LU: error term |det|^2 er2 + zabs2 as bfloat16 rounded up;
                            // the sign bit set marks a determinant redone in D64
    double2* D64;           // FP64 LU: det
};

// Index of the determinant of pattern z (of 2^r) for bitstring column col in
// D32 / E32 / D64: bitstring-major, so one bitstring's 2^r determinants are
// contiguous (coalesced reads by the combine; the LU's threads each write a
// run of consecutive patterns).
__host__ __device__ inline size_t dix(int64_t col, uint32_t z, int r) { return ((size_t)col << r) + z; }

// amp(b) = sum_{x_sh} WS[x_sh] prod_B A_B(x_sh),
// A_B(x_sh) = sum_{z < 2^r_loc} Omega_B[z] det_B(z ^ s_B[x_sh]).
struct ExactCombineDev {
    int nblocks;
    int k_sh;                       // bits of the gates shared by the two blocks
    uint64_t inactive0, inactive1;  // modes outside every active block (must be empty)
    uint64_t mask[kMaxBlocks][2];
    int eta[kMaxBlocks];
    int r[kMaxBlocks], r_loc[kMaxBlocks];
    const float2* D32[kMaxBlocks];
    const uint16_t* E32[kMaxBlocks];
    const double2* D64[kMaxBlocks];
    int src;                           // determinants from D32 (0), D64 (1), D32 with D64 where marked (2)
    const double2* Omega[kMaxBlocks];  // 2^r_loc pattern weights of the local gates
    const uint32_t* s[kMaxBlocks];     // 2^k_sh: pattern of the shared bits
    const uint32_t* perm[kMaxBlocks];  // shared bit patterns x_sh grouped by s >> r_loc
    const uint32_t* goff[kMaxBlocks];  // 2^(r - r_loc) + 1 group offsets
    const double2* WS;                 // 2^k_sh weights of the shared gates
    const float2* Omega32[kMaxBlocks]; // FP32 copies for the error estimate
    const double2* OmegaHat[kMaxBlocks];  // 2^r_loc: Walsh-Hadamard transform of Omega times 2^-r_loc
    const float4* OmegaHatDF[kMaxBlocks]; // the same as float pairs (re hi, im hi, re lo, im lo)
    const float4* WSDF;                   // WS as float pairs
    int wht;                           // 1: XOR convolutions by transforms in shared memory
    int wreg;                          // 1: transforms over FP32 determinants in registers
                                       //    (5 <= r <= 10 and 1 <= r_loc <= 5 in both blocks)
    int inj;                           // 1: every s_B is one-to-one
    const uint32_t* inv_off[kMaxBlocks];  // 2^r + 1: x_sh with s_B(x_sh) = z are
    const uint32_t* inv_xs[kMaxBlocks];   //   inv_xs[inv_off[z] .. inv_off[z + 1])
    const float2* WS32;
    double err_coef;                   // K u32 (FP32 path), 0 for FP64
    double tol, p_floor;
    int64_t minors;                    // determinants per bitstring, sum over blocks of 2^r
    int col_by_index;                  // D column of a listed bitstring: its index (1) or list position (0)
    // EF_PREC_AUTO: when flagging a result, list its determinants whose
    // variance terms are large (mlist[B] entries (column, z), counts in mcount)
    int2* mlist[kMaxBlocks];
    int* mcount;
    // recompute counters: [0] bitstrings, [1] FP64 determinants; the launch adds
    // the list size (count_bits), list size x minors (count_full), sum of mcount (count_minors)
    unsigned long long* recomp;
    int count_bits, count_full, count_minors;
};

// ---------------------------------------------------------------- Raw Estimate

struct ApproxBlockDev {
    int n, eta, L;
    uint64_t mask0, mask1;
    const void* P;    // interval products Pi_{a..b}, a >= b, tri index a(a+1)/2 + b, n x n each (path precision)
    const void* RC;   // L x n x eta: Pi_{l..0}[:, C] for l = 0..L-1 (path precision)
    const double2* P64;   // FP64 copies (prologue: A0, its inverse, K)
    const double2* RC64;
    const int* cols;  // eta local column indices
    int f;                // flippable (layer, mode) pairs of the block (<= 64)
    const int* pair_lm;   // [f]: (layer 1..L) << 8 | local mode, layer-major
};

struct ApproxDev {
    int nblocks;
    int k;
    const uint32_t* T;       // thresholds
    const double* qratio;    // (s/pT1) / (c/pT0) per gate
    const float* qratio32;   // the same in FP32 (FP32 path)
    const uint8_t* glayer;   // [kMaxBlocks][k]: layer 1..L in the block, 0 = not touching
    const uint64_t* gmodes;  // [kMaxBlocks][k]: local modes flipped in the block
    const uint64_t* gpair;   // [kMaxBlocks][k]: flippable pairs flipped in the block (K form)
    double R0;               // prod_j c_j / pT0_j
    uint32_t key0, key1;
    uint64_t index_base;
    const uint64_t* gidx;    // null: bitstring i has global index index_base + i; else gidx[i]
    uint64_t inactive0, inactive1;
    int64_t t;
    int64_t nb;              // bitstrings of the call
    const int* list;         // null: every bitstring; else the listed bitstrings (FP64 redo)
    const int* list_count;   //   their number (device)
    int traj_per_cta;
    int n_chunks;
    int grid;                // CTAs (grid-stride over (bitstring, chunk) items)
    int kform;               // 1: trajectory minors through K (every block has <= 64 flippable pairs)
    double kappa_max;        // A0 with ||A0||_1 ||A0^-1||_1 above this takes the rank-one form
    double err_coef;         // FP32 error estimate: K u32 (0: no estimate)
    double err_lin;          // FP32 error estimate, rank-one form: u32 (0: no estimate)
    double nmax;             // upper estimate of how many of the t trajectories share one rounded quantity
    double tol, p_floor;     // EF_PREC_AUTO threshold on the estimated relative error of p_hat
    double* part;                 // [nb][n_chunks][kApproxPartStride]
    unsigned long long* counters; // [0] flips, [1] executed eta x eta LUs, [2] rank-one-form minors, [3] flagged
    ApproxBlockDev blk[kMaxBlocks];
};

// One (circuit, mode block) of a multi-circuit FP32 LU work queue. Items are
// (bitstring tile of 128, chunk of patterns); entry e owns items
// [item_begin, item_begin + tiles * blk.n_chunks).
struct QueueEntry {
    ExactBlockDev blk;
    const uint64_t* bits;
    int64_t nb;
    int64_t tiles;
    int64_t item_begin;
};

// ---------------------------------------------------------------- adjoint

struct GradDev {
    ExactCombineDev cm;             // forward tables (D holds FP64 determinants)
    ExactBlockDev blk[kMaxBlocks];  // FP64 branch matrices, layer tables
    double2* cot[kMaxBlocks];       // [2^r][nb]: gamma_b d amp_b / d det_B(b, z)
    double2* ebar[kMaxBlocks];      // [nb][2^r_loc]: gamma_b d amp_b / d Omega_B(z)
    double2* pbar;                  // [nb][2^k_sh]: gamma_b d amp_b / d w_sh(x_sh)
    double2* tbar[kMaxBlocks];      // [2^r][L][n][n]: per-pattern d L / d T_l
    double2* sbar[kMaxBlocks];      // [2^r][n][eta]: per-pattern d L / d S_0[:, C]
};

// ---------------------------------------------------------------- launchers

struct LaunchStats {
    int64_t launches = 0;
    int64_t executed_lus = 0;
};

// Streaming multiprocessors of the current device (queried once per device;
// grids are sized in multiples of it).
int sm_count();

// Raise the kernel's dynamic shared-memory limit on the current device to at
// least `bytes`; it is never lowered. The limit is a property of the kernel,
// not of a launch: lowering it for a small launch would invalidate a larger
// launch of the same kernel recorded earlier in a CUDA graph (a replay that
// re-checks each node against the current limit then fails that node).
cudaError_t raise_dynamic_smem(const void* kernel, size_t bytes);

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel on the stream is still finishing, which hides the
// launch latency between the dependent kernels of a call. Every kernel
// launched this way calls cudaGridDependencySynchronize() before its first
// global-memory access, so it still sees all of the previous kernel's writes
// (and writes nothing the previous kernel reads) exactly as with an ordinary
// launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// branch matrices of nblk (1 or 2) mode blocks in one launch
cudaError_t launch_build_branches(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk, bool want32,
                                  cudaStream_t s, LaunchStats& st);
// FP32 minors of nblk (1 or 2) mode blocks with the same eta in one launch
cudaError_t launch_exact_lu_f32(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk, const uint64_t* bits,
                                int64_t nb, cudaStream_t s, LaunchStats& st);
// largest pattern count (log2) a chunk of the FP32 kernel can stage in shared memory
int exact_f32_chunk_log2(int n, int eta, int r, int64_t nb);
// Persistent FP32 LU over a work queue of several circuits with the same eta:
// CTAs take items from *head (reset to 0 before the launch) until none is left.
cudaError_t launch_queue_lu_f32(int eta, const QueueEntry* entries, int n_entries, int64_t n_items,
                                unsigned long long* head, size_t smem, int grid, cudaStream_t s,
                                LaunchStats& st);
// FP64 minors; thread per minor for eta <= 8, warp-row above
cudaError_t launch_exact_lu_f64(const ExactBlockDev& b, const uint64_t* bits, int64_t nb,
                                const int* list, const int* list_count, int64_t cap,
                                cudaStream_t s, LaunchStats& st);
// Float-pair (about 48-bit) redo of the listed determinants
// mlist_B[0..mcount[B]) of nblk blocks with the same eta (<= 16), in one launch
cudaError_t launch_exact_lu_redo_minors(const ExactBlockDev& b0, const ExactBlockDev& b1, int nblk,
                                        const uint64_t* bits, const int2* mlist0, const int2* mlist1,
                                        const int* mcount, cudaStream_t s, LaunchStats& st);
cudaError_t launch_exact_lu_rows(const ExactBlockDev& b, const uint64_t* bits, int64_t nb,
                                 const int* list, const int* list_count, int64_t cap,
                                 bool fp64, cudaStream_t s, LaunchStats& st);
size_t exact_combine_smem(const ExactCombineDev& c);
cudaError_t launch_exact_combine(const ExactCombineDev& c, const uint64_t* bits, int64_t nb, int64_t stride,
                                 const int* list, const int* list_count, double* out, double* err,
                                 int* append_list, int* append_count, cudaStream_t s, LaunchStats& st);
cudaError_t launch_grad(const GradDev& g, const uint64_t* bits, int64_t nb, const double* grad_p,
                        double* out_p, cudaStream_t s, LaunchStats& st);
size_t grad_minors_smem(int n, int eta, int L);
cudaError_t launch_sum_rows(const double2* in, int64_t count, int64_t stride, int64_t width, double2* out,
                            cudaStream_t s, LaunchStats& st);
// Raw Estimate: dynamic shared memory of one CTA; the launch over the items
// (all bitstrings, or a.list); the per-bitstring finalisation (listed: the
// FP64 redo of the listed bitstrings; append_list collects flagged ones)
size_t approx_smem_bytes(const ApproxDev& a, int eta_t, bool fp64);
int approx_eta_template(const ApproxDev& a);
cudaError_t launch_approx(const ApproxDev& a, const uint64_t* bits, bool fp64, cudaStream_t s, LaunchStats& st);
cudaError_t launch_approx_finalize(const ApproxDev& a, double* out, double* stderr_out, double* err_out,
                                   int* append_list, int* append_count, bool listed, cudaStream_t s,
                                   LaunchStats& st);

}  // namespace ef
