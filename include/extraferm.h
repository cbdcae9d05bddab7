/*
 * extraferm.h -- C ABI of a GB300 (sm_103a) engine for Born-rule probabilities
 * of bitstrings under particle-number-conserving extended matchgate circuits:
 * nearest-neighbour Givens rotations and single-mode phases (passive
 * matchgates, Section II-B, Eqs. 1-3) plus k controlled-phase gates
 * (Section III-B, Eq. 7).
 *
 * The method (Section III-A/B):
 *   - each controlled-phase gate c(theta) is the weighted sum
 *     e^{i theta/4}[cos(theta/4) d0(theta) + i sin(theta/4) d1(theta)] of two
 *     passive gates (Eq. 7); a trajectory x in {0,1}^k picks one term per gate;
 *   - for a trajectory the circuit is passive with an n x n mode-transformation
 *     matrix V(x), and <b|V(x)|a> is the eta x eta minor of V(x) with rows the
 *     set bits of b and columns the set bits of a (Terhal-DiVincenzo, Eq. 3);
 *   - Exact (Eqs. 8-9): p(b) = |sum_x w(x) <b|V(x)|a>|^2 over all 2^k
 *     trajectories, w(x) = prod_j cos(theta_j/4)^{1-x_j} (i sin(theta_j/4))^{x_j};
 *   - Raw Estimate (Eqs. 10-12, Section III-A): t trajectories drawn from
 *     P(x) = prod_j p(x_j), p(x_j = 1) = sin(|theta_j|/4)/(sin + cos), and
 *     p_hat = |(1/t) sum_s w(x_s)/P(x_s) <b|V(x_s)|a>|^2.
 *
 * Conventions.
 *   - Modes 0..n-1 (n <= 128). Bit m of a bitstring is the occupation of mode
 *     m; a bitstring is two little-endian 64-bit words (word 0 = modes 0..63).
 *     Bitstring arrays are nb x 2 uint64, row-major.
 *   - Gate matrices act on the single-particle space in the column convention:
 *     a circuit's matrix is the product of its gates' matrices with later gates
 *     on the left.
 *       EF_GIVENS (p, q = p+1, theta, phi):
 *         [[cos theta, -e^{i phi} sin theta], [e^{-i phi} sin theta, cos theta]]
 *         on modes (p, q);
 *       EF_PHASE (p, phi): mode p gets e^{i phi} (q ignored);
 *       EF_CPHASE (p != q, theta): diag(1, 1, 1, e^{i theta}) on the qubits of
 *         modes p and q (any pair, not only neighbours).
 *   - Controlled-phase angles are used modulo 2 pi, wrapped to (-pi, pi].
 *   - A bitstring whose Hamming weight (or, when the circuit splits into
 *     independent mode blocks, whose weight inside a block) differs from the
 *     initial state's gets probability 0 exactly; that is not an error.
 *     A bit at or above n_modes is: the host-pointer calls return EF_EINVAL
 *     and leave the outputs untouched (the *_dev calls do not inspect the
 *     bits on the host; the kernels read them only through the circuit's
 *     mode masks).
 *   - Angles: the differentiable angle vector lists, per gate in circuit order,
 *     Givens -> (theta, phi), PHASE -> phi, CPHASE -> theta.
 *
 * Errors. Every call returns EF_OK (0) or a negative ef_status and never
 * aborts; ef_last_error() gives a message for the calling thread's last
 * failure. Host-pointer calls are synchronous. The *_dev calls take device
 * pointers and a cudaStream_t (passed as void*), enqueue their work on that
 * stream and return without waiting (except ef_prob_grad_dev, see there).
 *
 * Ownership and threading. ef_circuit_create copies the gate list; the
 * caller owns every input and output buffer. A circuit owns its device
 * tables and a grow-only device workspace, so the calls on one circuit must
 * be ordered (one host thread at a time, one stream at a time); different
 * circuits are independent.
 */
#ifndef EXTRAFERM_H
#define EXTRAFERM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ef_circuit ef_circuit; /* opaque, library-owned */

typedef enum {
    EF_OK = 0,
    EF_EINVAL = -1,        /* bad argument: null pointer, bad gate, bit >= n, ... */
    EF_ENOMEM = -2,        /* host or device allocation failed */
    EF_ECUDA = -3,         /* a CUDA runtime call failed (message has the CUDA error) */
    EF_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    EF_EUNSUPPORTED = -5   /* valid input outside what this build implements */
} ef_status;

typedef enum { EF_GIVENS = 0, EF_PHASE = 1, EF_CPHASE = 2 } ef_gate_kind;

typedef struct {
    int32_t kind;     /* ef_gate_kind */
    int32_t p, q;     /* modes */
    int32_t reserved; /* must be 0 */
    double theta;     /* GIVENS, CPHASE */
    double phi;       /* GIVENS, PHASE */
} ef_gate;            /* 32 bytes */

typedef enum {
    EF_PREC_FP64 = 0,       /* minors, LU and accumulation in FP64 */
    EF_PREC_FP32_MINOR = 1, /* minors and LU in FP32; Exact branch sums in float-pair
                               arithmetic (about 48 bits); Raw Estimate: per-bitstring
                               tables (A0, its inverse, K) in FP64, trajectory terms
                               in FP32 summed in float pairs */
    EF_PREC_AUTO = 2        /* FP32 minors; Exact: for results whose error estimate
                               exceeds tol the determinants carrying most of the
                               estimated error are redone in float-pair arithmetic
                               (about 48 bits, on the FP32 pipes; at most 8 particles
                               per block), then the result is re-estimated and, if
                               still above tol, all of its determinants are redone
                               in FP64; Raw Estimate: such results are recomputed
                               in FP64 */
} ef_precision;

enum {
    EF_FLAG_TIME_KERNELS = 1 /* record CUDA events around the dominant kernel */
};

typedef struct {
    int32_t precision;         /* ef_precision; default EF_PREC_AUTO */
    int32_t flags;             /* EF_FLAG_* */
    double tol;                /* relative-error target of EF_PREC_AUTO, default 1e-5 */
    int32_t tile_override[4];  /* 0 = automatic; [0] = FP32 Exact flip patterns per chunk (log2);
                                  [1] = constant K of the FP32 error estimate in tenths (default 40) */
} ef_options;

typedef struct {
    int64_t logical_branch_dets;  /* (bitstring, branch or trajectory) pairs the call evaluated */
    int64_t executed_minor_lus;   /* LU factorizations of minors actually run */
    int64_t fp64_recomputed;      /* EF_PREC_AUTO: flagged bitstrings, whose largest-error determinants
                                     were redone in float pairs (or, if still above tol, all of them in
                                     FP64) (Exact), or which were recomputed in FP64 (Raw Estimate); the
                                     redone determinants are counted in executed_minor_lus */
    int64_t kernel_launches;      /* kernels this library launched in the call */
    int64_t sampled_flips;        /* Raw Estimate: number of x_j = 1 over all trajectories */
    double max_est_rel_err;       /* largest per-result error estimate of the FP32 path */
    double dominant_kernel_ms;    /* device time of the dominant kernel (EF_FLAG_TIME_KERNELS) */
    int64_t dominant_kernel_launches;
    double dominant_kernel_flops; /* algorithmic flops of those launches */
} ef_stats;

/* Library version (major*10000 + minor*100 + patch). */
int ef_version(void);

/* Message of the calling thread's last error ("" if none). Valid until the
 * thread's next failing call. */
const char* ef_last_error(void);

/* Create a circuit on n_modes modes (1..128) with the initial basis state
 * `occupation` (2 words, bit m = mode m occupied, no bit >= n_modes) and the
 * gate list `gates[0..n_gates)` in circuit order. `opt` may be NULL for the
 * defaults. Host preprocessing (Section IV-A: per-gate sin/cos tables
 * computed once): angle wrapping, weight and sampling-threshold tables,
 * detection of independent mode blocks (modes joined by Givens rotations),
 * and the FP64 segment matrices between runs of controlled-phase gates
 * (Section IV-B, Eq. 14). Uses the current CUDA device. */
int ef_circuit_create(int32_t n_modes, const uint64_t occupation[2], const ef_gate* gates,
                      int64_t n_gates, const ef_options* opt, ef_circuit** out);

/* Release a circuit and its device memory (waits for its pending work). NULL is allowed. */
int ef_circuit_destroy(ef_circuit* c);

/* Number of differentiable angles (see Conventions). */
int ef_circuit_num_angles(const ef_circuit* c, int64_t* n);

/* Copy the angle vector out / replace it (n must equal the count) and redo
 * the host preprocessing. */
int ef_circuit_get_angles(const ef_circuit* c, double* angles, int64_t n);
int ef_circuit_set_angles(ef_circuit* c, const double* angles, int64_t n);

/* Extent xi* = prod_j (cos(|theta_j|/4) + sin(|theta_j|/4))^2 (Eq. 5). */
int ef_circuit_extent(const ef_circuit* c, double* xi);

/* Change the precision mode and tolerance of later calls. */
int ef_circuit_set_precision(ef_circuit* c, int32_t precision, double tol);

/* Exact algorithm (Eqs. 8-9) for bitstrings bits[0..nb) (host, nb x 2 uint64).
 * out[nb]: probabilities. err_out[nb] (nullable): per-result estimate of the
 * relative error of the FP32-minor path (0 on the FP64 path; for results
 * redone under EF_PREC_AUTO, the FP32 estimate that triggered it,
 * negated). nb = 0 is allowed. The circuit's 2^k trajectories are enumerated
 * per independent mode block as distinct flip patterns; controlled-phase
 * gates whose modes no Givens rotation touches before them, or after them,
 * change no probability and are left out. EF_EUNSUPPORTED beyond 2^22 flip
 * patterns, 22 enumerated controlled-phase gates or 32 particles in a mode
 * block, or 12 controlled-phase gates shared by two blocks. */
int ef_prob_exact(ef_circuit* c, const uint64_t* bits, int64_t nb, double* out, double* err_out);
int ef_prob_exact_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, double* d_out,
                      double* d_err_out, void* stream);

/* Raw Estimate (Eqs. 10-12) with n_traj trajectories per bitstring.
 * Trajectory s of bitstring i draws, for gate j, the 32-bit word (j mod 4) of
 * Philox4x32-10 with counter (j/4, s, g_lo, g_hi) and key (seed_lo, seed_hi),
 * g = index_base + i (the bitstring's global index), and sets x_j = 1 iff the
 * word is below T_j = round(p(x_j=1) 2^32) (>= 1 when sin(theta_j/4) != 0).
 * Importance weights use the quantised probabilities T_j/2^32, so the
 * amplitude estimate is unbiased. out[nb]: p_hat = |alpha_hat|^2;
 * stderr_out[nb] (nullable): 2 sqrt(Var_s[Re(conj(alpha_hat) Y_s)] / t).
 * A trajectory's minor is evaluated as det A0 * det(I + K[N, N]) with A0 the
 * bitstring's no-flip minor and K built once per bitstring in FP64 over the
 * (layer, mode) pairs a gate can flip (Section IV-B, Eqs. 15-18); more than
 * four flipped pairs in a block, or an ill-conditioned A0, take an eta x eta
 * LU of the rank-one-updated minor instead.
 * err_out[nb] (nullable): estimated relative error of p_hat, the rounding of
 * the FP32 path against the same estimator in exact arithmetic (0 on the FP64
 * path). Under EF_PREC_AUTO bitstrings whose
 * estimate exceeds tol are recomputed in FP64 with the same trajectories and
 * their err_out is the triggering estimate, negated. */
int ef_prob_approx(ef_circuit* c, const uint64_t* bits, int64_t nb, int64_t n_traj, uint64_t seed,
                   uint64_t index_base, double* out, double* stderr_out, double* err_out);
int ef_prob_approx_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, int64_t n_traj,
                       uint64_t seed, uint64_t index_base, double* d_out, double* d_stderr_out,
                       double* d_err_out, void* stream);

/* Estimate (Section III-A): |out[i] - p_i| <= eps for every bitstring, each
 * with failure probability at most delta (Eq. 6's guarantee), without a
 * given bound p_max. Rounds r = 0 .. R-1 of Raw Estimate on all bitstrings
 * (host arrays, synchronous): eps_r = max(eps, eps_0 / 2^r) with
 * eps_0 = max(eps, 1/4) and R the first round with eps_r = eps, failure
 * budget delta / R per round, and for each bitstring the Eq. 6 trajectory
 * count for its own bound p_max (1 in round 0, then min(p_max, p_hat + eps_r)
 * of the previous round), rounded up to m 2^e with 4 <= m <= 8 so that equal
 * counts share a launch. Round r draws with seed splitmix64(seed +
 * (r + 1) 0x9E3779B97F4A7C15) and the bitstrings' global indices
 * index_base + i (as ef_prob_approx). out: the last round's p_hat;
 * stderr_out, traj_out (nullable): its standard error and the total
 * trajectories spent per bitstring. Bitstrings outside the particle sector
 * get 0 with no trajectories. EF_EUNSUPPORTED if a round needs more than
 * 2^32 trajectories for a bitstring. */
int ef_prob_estimate(ef_circuit* c, const uint64_t* bits, int64_t nb, double eps, double delta,
                     uint64_t seed, uint64_t index_base, double* out, double* stderr_out,
                     int64_t* traj_out);

/* Vector-Jacobian product of the Exact probabilities: grad_angles[j] =
 * sum_b grad_p[b] * d p_b / d angle_j for every angle of the angle vector
 * (FP64). out_p (nullable) receives the probabilities. The device kernels
 * reduce the cotangents to per-segment matrices; the chain rule through the
 * individual gates runs on the host, so ef_prob_grad_dev, unlike the other
 * *_dev calls, waits for its stream before it returns (d_grad_angles is
 * written by then). */
int ef_prob_grad(ef_circuit* c, const uint64_t* bits, int64_t nb, const double* grad_p,
                 double* out_p, double* grad_angles);
int ef_prob_grad_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, const double* d_grad_p,
                     double* d_out_p, double* d_grad_angles, void* stream);

/* Exact algorithm like ef_prob_exact_dev, for callers that cannot let a
 * library allocate GPU memory while they run: for example a service that
 * hands all device memory to its own pool at start-up (a later cudaMalloc
 * would fail or evict its data), or a latency-bound loop in which a
 * cudaMalloc/cudaFree would synchronise the device and stall other streams.
 * The paper has no counterpart; this is an interface of this library.
 *
 * Everything the call needs on the device (circuit tables, branch
 * matrices, partial sums, the recompute list) is carved from one fixed
 * 64 MiB array declared at file scope in the library, which every GPU that
 * loads the library holds until the process exits. The call itself performs
 * no cudaMalloc, cudaFree or other allocating call; the caller still passes
 * the bitstrings and outputs (device pointers). The first call on a device
 * looks the array's device address up (cudaGetSymbolAddress with that device
 * current); make that first call before any stream capture. The circuit's
 * tables sit at the start of the array: a call copies them in from host
 * memory (ordinary cudaMemcpyAsync from pageable memory) unless the previous
 * call on this device was on the same circuit with the same angles, in which
 * case it finds them in place and copies nothing. A call that copies cannot
 * be captured in a CUDA graph (pageable copies are not allowed in a capture);
 * a call that finds the tables in place, on the stream of the circuit's
 * previous call, copies, synchronises and allocates nothing and can be
 * captured and replayed (the tests capture one). Calls whose tables, branch
 * matrices and per-bitstring partials do not fit return EF_EINVAL with the
 * largest batch that fits; split the batch. All calls (on any circuit and
 * any stream) share the array and it keeps the last call's contents, so
 * calls that overlap on the GPU race: order them on one stream or
 * synchronise between them. The circuit's stats of the call are available
 * from ef_circuit_get_stats (no kernel timing); under EF_PREC_AUTO its FP64
 * recompute counts are read from the array, so they are valid only until
 * the next allocation-free call on the same device. */
int ef_prob_exact_noalloc_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, double* d_out,
                              double* d_err_out, void* stream);

/* ---- Multi-circuit batch (no counterpart in the paper; Section IV-A runs
 * one circuit at a time). A batch evaluates many circuits of uneven modes,
 * particles and controlled-phase gates in one CUDA graph: Exact circuits
 * with FP32 minors share persistent work-queue LU kernels (one per particle
 * count) whose chunk sizes are chosen on first use by timing; Raw Estimate
 * circuits and the per-circuit sums run on forked streams. The batch does
 * not own the circuits; destroy it before them. */
typedef struct ef_batch ef_batch;

/* Create a batch over circuits cs[0..nc). A circuit may appear once
 * (EF_EINVAL otherwise): its workspace holds one evaluation at a time. */
int ef_batch_create(ef_circuit* const* cs, int32_t nc, ef_batch** out);

/* Release a batch (waits for its work). NULL is allowed. */
int ef_batch_destroy(ef_batch* b);

/* Probabilities of every circuit of the batch. All arrays are host arrays
 * of length nc: d_bits[i] (device, nb[i] x 2 uint64) and d_out[i] (device,
 * nb[i] doubles) for circuit i; n_traj[i] = 0 selects the Exact algorithm
 * (in the circuit's precision mode), n_traj[i] > 0 the Raw Estimate with
 * that many trajectories (seed `seed`, global bitstring indices 0..nb[i]-1).
 * The first call with a given set of arguments plans, runs and captures the
 * work (synchronous); later calls with the same arguments replay the graph on
 * `stream` (asynchronous). Changing a circuit's angles re-plans, and so does
 * a call on one of the circuits outside the batch that had to enlarge the
 * circuit's device workspace (the graph holds its addresses). */
int ef_batch_prob_dev(ef_batch* b, const uint64_t* const* d_bits, const int64_t* nb, double* const* d_out,
                      const int64_t* n_traj, uint64_t seed, void* stream);

/* Kernel launches of one batch execution and the logical branch count. */
int ef_batch_get_stats(ef_batch* b, ef_stats* st);

/* Counters and timings of the circuit's last probability call (waits for it). */
int ef_circuit_get_stats(ef_circuit* c, ef_stats* st);

/* Measured throughput of the current GPU, for roofline denominators (the
 * paper has no counterpart): kind 0 = FP32 FMA flops/s (scalar FFMA), 1 = FP32
 * FMA flops/s (packed FFMA2), 2 = FP64 FMA flops/s, 3 = Philox4x32-10 blocks/s.
 * Independent dependency chains in every lane of 8 CTAs per SM; best of `reps`
 * timed launches after one warm-up; synchronous; allocates a small buffer. */
int ef_measure_peak(int32_t kind, int32_t reps, double* rate);

#ifdef __cplusplus
}
#endif

#endif /* EXTRAFERM_H */
