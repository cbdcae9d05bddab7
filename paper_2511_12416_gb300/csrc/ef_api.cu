// Host runtime and C ABI (include/extraferm.h).
//
// Host preprocessing in FP64 (Section IV-A: sin/cos tables precomputed once):
//   * controlled-phase tables: wrapped angle, c = cos(theta/4), s = sin(theta/4)
//     (Eq. 7), sampling threshold T = round(p(x=1) 2^32) (Eqs. 10-12);
//   * independent mode blocks: modes joined by Givens rotations; at most two
//     blocks holding particles are kept apart (more are merged into one);
//   * per block, the passive segments S_0..S_L between the runs of
//     controlled-phase gates that touch the block, and T_l = S_l diag(base
//     phases e^{i theta/2} of layer l) (Section IV-B, Eqs. 14-18);
//   * Exact: GF(2) basis of the blocks' flip patterns, pattern flip masks,
//     pattern weights of the local gates and the shared-gate tables;
//   * Raw Estimate: interval products Pi_{a..b} = T_a ... T_b.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <map>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ef_internal.h"
#include "extraferm.h"

using cd = std::complex<double>;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define EF_CK(call)                                                                              \
    do {                                                                                         \
        cudaError_t _e = (call);                                                                 \
        if (_e != cudaSuccess)                                                                   \
            return fail(EF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));           \
    } while (0)

constexpr double kTwo32 = 4294967296.0;
constexpr double kPi = 3.14159265358979323846;

double wrap_angle(double theta) {
    double t = theta - 2.0 * kPi * std::floor((theta + kPi) / (2.0 * kPi));
    if (t <= -kPi) t += 2.0 * kPi;
    return t;
}

struct CP {
    int gate, p, q;
    double theta, c, s, pT0, pT1, ratio0, ratio1;
    uint32_t T;
    int blk_p, blk_q;  // active block of each mode (-1 = none)
    int cls;           // -1 outside the Exact enumeration, 0/1 local to block, 2 shared
    bool phase_only;   // changes no probability (see the gate classes in prepare)
};

// A device buffer that only grows. Every reallocation bumps the owner's
// workspace epoch, so that captured work holding the old address can tell.
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    uint64_t* epoch = nullptr;
    cudaError_t ensure(size_t want) {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (epoch) ++*epoch;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(want, 256));
        if (e == cudaSuccess) bytes = std::max<size_t>(want, 256);
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

template <typename T>
cudaError_t upload(DBuf& d, const std::vector<T>& h, cudaStream_t s) {
    cudaError_t e = d.ensure(h.size() * sizeof(T));
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// complex values as float pairs (re hi, im hi, re lo, im lo), hi + lo = value to ~48 bits
std::vector<float4> to_ff(const std::vector<cd>& v) {
    std::vector<float4> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float rh = (float)v[i].real(), ih = (float)v[i].imag();
        o[i] = make_float4(rh, ih, (float)(v[i].real() - (double)rh), (float)(v[i].imag() - (double)ih));
    }
    return o;
}

struct HostBlock {
    int n = 0, eta = 0, L = 0;
    uint64_t mask[2] = {0, 0};
    std::vector<int> modes;  // local -> global
    std::vector<int> cols;   // occupied local modes
    std::vector<std::vector<int>> layers;  // cphase indices per layer (1..L -> [0..L-1])
    std::vector<std::vector<int>> seg_gates;  // gate indices of segment l (0..L), in circuit order
    std::vector<int> local_of;                // global mode -> local index (-1 outside)
    std::vector<cd> S;       // (L+1) n x n segments
    std::vector<cd> T;       // (L+1) n x n: T_0 = S_0, T_l = S_l diag(D_l0)
    // Exact
    int k_loc = 0;
    std::vector<int> local_gates;  // cphase indices local to the block
    int r = 0, r_loc = 0;          // rank of the flip patterns / of the local gates' patterns
    int r_sign = 0;                // rank of the patterns of gates that only change minors' signs
    std::vector<uint32_t> F;       // L x n: flip masks over pattern bits
    std::vector<cd> Omega;         // 2^r_loc: weights of the local gates folded onto patterns
    std::vector<float2> Omega32;   // FP32 copy (error estimate)
    std::vector<cd> OmegaHat;      // Walsh-Hadamard transform of Omega over the r_loc bits, times 2^-r_loc
    std::vector<float4> OmegaHatFF;  // the same as float pairs
    std::vector<uint32_t> sh;      // 2^k_sh: pattern of each shared bit vector
    std::vector<uint32_t> perm, goff;  // shared bit vectors grouped by pattern >> r_loc
    std::vector<uint32_t> inv_off, inv_xs;  // shared bit vectors grouped by pattern
    std::vector<uint32_t> coord;       // pattern coordinates of the local, then shared gates
    int c_log2 = 0;
    // Raw Estimate
    std::vector<cd> P;   // tri(L) x n x n
    std::vector<cd> RC;  // L x n x eta
    std::vector<int> pair_lm;  // flippable (layer, mode) pairs, layer-major: layer << 8 | local mode
    // device
    DBuf dS0C, dT, dF, dOmega, dOmega32, dOmegaHat, dOmegaHatFF, dSh, dPerm, dGoff, dInvOff, dInvXs, dM64, dM32, dD32, dE32, dD64, dMlist,
        dP64, dP32, dRC64, dRC32, dCols, dPairLM;
    DBuf dCot, dEbar, dTbar, dSbar, dSumT, dSumS, dSumE;
    template <typename F> void for_each_buf(F f) {
        for (DBuf* b : {&dS0C, &dT, &dF, &dOmega, &dOmega32, &dOmegaHat, &dOmegaHatFF, &dSh, &dPerm, &dGoff, &dInvOff, &dInvXs, &dM64, &dM32, &dD32, &dE32, &dD64, &dMlist, &dP64, &dP32, &dRC64,
                        &dRC32, &dCols, &dPairLM, &dCot, &dEbar, &dTbar, &dSbar, &dSumT, &dSumS, &dSumE})
            f(*b);
    }
    void release() {
        for_each_buf([](DBuf& b) { b.release(); });
    }
};

int tri(int a, int b) { return a * (a + 1) / 2 + b; }

double log_binom(int n, int k) { return std::lgamma(n + 1.0) - std::lgamma(k + 1.0) - std::lgamma(n - k + 1.0); }

}  // namespace

struct ef_circuit {
    int n = 0;
    uint64_t occ[2] = {0, 0};
    std::vector<ef_gate> gates;
    ef_options opt{};
    int device = 0;

    // derived
    std::vector<CP> cps;
    double xi = 1.0;
    int nblocks = 0;
    HostBlock blk[ef::kMaxBlocks];
    uint64_t inactive[2] = {0, 0};
    std::vector<int> shared_gates;
    std::vector<cd> WS;  // 2^k_sh weights of the shared gates
    std::vector<float2> WS32;
    std::vector<float4> WSFF;  // WS as float pairs
    bool exact_ok = true;
    std::string exact_why;
    bool approx_ok = true;
    std::string approx_why;
    double p_floor = 0.0;
    // Raw Estimate gate tables
    std::vector<uint32_t> aT;
    std::vector<double> aq;
    std::vector<float> aq32;
    std::vector<uint8_t> alayer;
    std::vector<uint64_t> amodes;
    std::vector<uint64_t> agpair;  // [kMaxBlocks][k]: flippable pairs each gate flips (K form)
    bool kform_ok = false;         // every block has at most 64 flippable pairs
    double R0 = 1.0;

    bool dirty = true;
    DBuf dWS, dWS32, dWSFF, dList, dListCount, dRecomp, dBits, dOut, dErr, dGradP, dGrad, dPbar, dSumP;
    DBuf daT, daq, daq32, dalayer, damodes, dagpair, daPart, dCounters, daList;
    cudaStream_t own_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    cudaStream_t last_stream = nullptr;
    bool has_last_stream = false;  // the legacy default stream is a null handle
    ef_stats stats{};
    int64_t last_fp64_list_pending = 0;  // 1 if the FP64 recompute count must be read back
    int64_t last_sub_total = 0;          // sum over blocks of 2^r (minors per bitstring)
    unsigned long long* last_recomp = nullptr;          // device counter of the last call's FP64 recomputes
    int last_mode = 0;                   // 1 exact, 2 approx

    uint64_t ws_epoch = 0;    // bumped whenever one of the circuit's device buffers is reallocated
    uint64_t uid = 0;         // process-unique id (addresses of destroyed circuits are reused)
    uint64_t tables_gen = 0;  // bumped by every host preprocessing (angles changed)

    template <typename F> void for_each_buf(F f) {
        for (int b = 0; b < ef::kMaxBlocks; ++b) blk[b].for_each_buf(f);
        for (DBuf* d : {&dWS, &dWS32, &dWSFF, &dList, &dListCount, &dRecomp, &dBits, &dOut, &dErr, &dGradP, &dGrad, &dPbar, &dSumP, &daT,
                        &daq, &daq32, &dalayer, &damodes, &dagpair, &daPart, &dCounters, &daList})
            f(*d);
    }
    ef_circuit() {
        for_each_buf([this](DBuf& d) { d.epoch = &ws_epoch; });
    }
    ~ef_circuit() {
        for_each_buf([](DBuf& d) { d.release(); });
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (own_stream) cudaStreamDestroy(own_stream);
    }
};

namespace {

// ------------------------------------------------------------------ preprocessing

int prepare(ef_circuit* c) {
    const int n = c->n;
    // controlled-phase tables
    c->cps.clear();
    c->xi = 1.0;
    for (size_t gi = 0; gi < c->gates.size(); ++gi) {
        const ef_gate& g = c->gates[gi];
        if (g.kind != EF_CPHASE) continue;
        CP cp{};
        cp.gate = (int)gi;
        cp.p = g.p;
        cp.q = g.q;
        cp.theta = wrap_angle(g.theta);
        cp.c = std::cos(cp.theta / 4.0);
        cp.s = std::sin(cp.theta / 4.0);
        const double sa = std::sin(std::fabs(cp.theta) / 4.0), ca = std::cos(std::fabs(cp.theta) / 4.0);
        const double p1 = sa / (sa + ca);
        uint64_t T = 0;
        if (sa != 0.0) {
            T = (uint64_t)std::floor(p1 * kTwo32 + 0.5);
            T = std::min<uint64_t>(std::max<uint64_t>(T, 1), 4294967295ull);
        }
        cp.T = (uint32_t)T;
        cp.pT1 = (double)T / kTwo32;
        cp.pT0 = 1.0 - cp.pT1;
        cp.ratio0 = cp.c / cp.pT0;
        cp.ratio1 = T > 0 ? cp.s / cp.pT1 : 0.0;
        c->xi *= (ca + sa) * (ca + sa);
        c->cps.push_back(cp);
    }
    const int k = (int)c->cps.size();

    // components joined by Givens rotations (adjacent modes -> intervals)
    std::vector<int> comp(n);
    {
        std::vector<char> join(n, 0);  // join[m]: m and m+1 connected
        for (const ef_gate& g : c->gates)
            if (g.kind == EF_GIVENS) join[g.p] = 1;
        int id = 0;
        for (int m = 0; m < n; ++m) {
            comp[m] = id;
            if (!(m + 1 < n && join[m])) ++id;
        }
    }
    const int ncomp = comp[n - 1] + 1;
    std::vector<int> comp_eta(ncomp, 0);
    for (int m = 0; m < n; ++m)
        if ((c->occ[m >> 6] >> (m & 63)) & 1ull) comp_eta[comp[m]]++;
    std::vector<int> active;
    for (int i = 0; i < ncomp; ++i)
        if (comp_eta[i] > 0) active.push_back(i);
    std::vector<int> block_of_comp(ncomp, -1);
    if (active.size() <= (size_t)ef::kMaxBlocks) {
        for (size_t i = 0; i < active.size(); ++i) block_of_comp[active[i]] = (int)i;
        c->nblocks = (int)active.size();
    } else {
        for (int a : active) block_of_comp[a] = 0;
        c->nblocks = 1;
    }
    std::vector<int> block_of(n), local_of(n, -1);
    c->inactive[0] = c->inactive[1] = 0;
    for (int b = 0; b < ef::kMaxBlocks; ++b) {
        HostBlock& B = c->blk[b];
        B.modes.clear();
        B.cols.clear();
        B.mask[0] = B.mask[1] = 0;
    }
    for (int m = 0; m < n; ++m) {
        const int b = block_of_comp[comp[m]];
        block_of[m] = b;
        if (b < 0) {
            c->inactive[m >> 6] |= 1ull << (m & 63);
            continue;
        }
        HostBlock& B = c->blk[b];
        local_of[m] = (int)B.modes.size();
        if ((c->occ[m >> 6] >> (m & 63)) & 1ull) B.cols.push_back(local_of[m]);
        B.modes.push_back(m);
        B.mask[m >> 6] |= 1ull << (m & 63);
    }
    for (int b = 0; b < c->nblocks; ++b) {
        c->blk[b].n = (int)c->blk[b].modes.size();
        c->blk[b].eta = (int)c->blk[b].cols.size();
    }
    // Controlled-phase gates that change no probability: each of their modes is
    // untouched by Givens rotations either before the gate (it still holds its
    // initial occupation, so the gate reduces to a phase on the other mode or to
    // a global phase) or after it (the gate, or that reduced phase, commutes with
    // everything later and ends as a diagonal gate before the measurement). Their
    // factor c + i s sigma in the amplitude (sigma = +-1, the sign their flips give
    // the minors) has modulus 1, so the Exact path leaves them out of its branch
    // enumeration (class -1 below) and their probability gradient is zero. The
    // Raw Estimate keeps them: its estimator samples every gate.
    std::vector<int> first_rot(n, (int)c->gates.size()), last_rot(n, -1);
    for (int gi = 0; gi < (int)c->gates.size(); ++gi) {
        const ef_gate& g = c->gates[gi];
        if (g.kind != EF_GIVENS) continue;
        for (int m : {g.p, g.q}) {
            first_rot[m] = std::min(first_rot[m], gi);
            last_rot[m] = std::max(last_rot[m], gi);
        }
    }
    // gate classes
    c->shared_gates.clear();
    for (int j = 0; j < k; ++j) {
        CP& cp = c->cps[j];
        cp.blk_p = block_of[cp.p];
        cp.blk_q = block_of[cp.q];
        auto settled = [&](int m) { return first_rot[m] > cp.gate || last_rot[m] < cp.gate; };
        cp.phase_only = settled(cp.p) && settled(cp.q);
        if ((cp.blk_p < 0 && cp.blk_q < 0) || cp.phase_only) cp.cls = -1;
        else if (cp.blk_p >= 0 && cp.blk_q >= 0 && cp.blk_p != cp.blk_q) cp.cls = 2;
        else cp.cls = cp.blk_p >= 0 ? cp.blk_p : cp.blk_q;
        if (cp.cls == 2) c->shared_gates.push_back(j);
    }
    const int k_sh = (int)c->shared_gates.size();

    c->exact_ok = true;
    c->exact_why.clear();
    c->approx_ok = true;
    c->approx_why.clear();
    double log_sector = 0.0;
    c->alayer.assign((size_t)ef::kMaxBlocks * k, 0);
    c->amodes.assign((size_t)ef::kMaxBlocks * k, 0);
    c->agpair.assign((size_t)ef::kMaxBlocks * k, 0);
    c->kform_ok = true;

    // per-block segments, layers and tables
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const int nb_ = B.n;
        log_sector += log_binom(B.n, B.eta);
        auto eye = [&]() {
            std::vector<cd> I((size_t)nb_ * nb_, cd(0, 0));
            for (int i = 0; i < nb_; ++i) I[(size_t)i * nb_ + i] = 1.0;
            return I;
        };
        std::vector<std::vector<cd>> segs;
        B.layers.clear();
        B.seg_gates.clear();
        std::vector<cd> seg = eye();
        std::vector<int> segg;  // gates of the current segment, in order
        bool in_layer = false;
        std::vector<int> cur;
        int j = 0;
        std::vector<int> layer_of_cp(k, 0);
        for (const ef_gate& g : c->gates) {
            const int gi = (int)(&g - c->gates.data());
            if (g.kind == EF_CPHASE) {
                const CP& cp = c->cps[j];
                const bool touches = cp.blk_p == b || cp.blk_q == b;
                if (touches) {
                    if (!in_layer) {
                        segs.push_back(seg);
                        B.seg_gates.push_back(segg);
                        in_layer = true;
                        cur.clear();
                    }
                    cur.push_back(j);
                    layer_of_cp[j] = (int)B.layers.size() + 1;
                }
                ++j;
                continue;
            }
            if (block_of[g.p] != b) continue;
            if (in_layer) {
                B.layers.push_back(cur);
                in_layer = false;
                seg = eye();
                segg.clear();
            }
            segg.push_back(gi);
            const int lp = local_of[g.p];
            if (g.kind == EF_GIVENS) {
                const int lq = local_of[g.q];
                const double ct = std::cos(g.theta), st = std::sin(g.theta);
                const cd e = std::polar(1.0, g.phi), em = std::polar(1.0, -g.phi);
                const cd g00 = ct, g01 = -e * st, g10 = em * st, g11 = ct;
                for (int col = 0; col < nb_; ++col) {
                    const cd a = seg[(size_t)lp * nb_ + col], bb = seg[(size_t)lq * nb_ + col];
                    seg[(size_t)lp * nb_ + col] = g00 * a + g01 * bb;
                    seg[(size_t)lq * nb_ + col] = g10 * a + g11 * bb;
                }
            } else {  // PHASE
                const cd e = std::polar(1.0, g.phi);
                for (int col = 0; col < nb_; ++col) seg[(size_t)lp * nb_ + col] *= e;
            }
        }
        if (in_layer) {
            B.layers.push_back(cur);
            seg = eye();
            segg.clear();
        }
        segs.push_back(seg);
        B.seg_gates.push_back(segg);
        B.L = (int)B.layers.size();
        const int L = B.L;
        const size_t nn = (size_t)nb_ * nb_;
        B.S.assign((size_t)(L + 1) * nn, cd(0, 0));
        B.T.assign((size_t)(L + 1) * nn, cd(0, 0));
        for (int l = 0; l <= L; ++l) std::copy(segs[l].begin(), segs[l].end(), B.S.begin() + l * nn);
        // T_0 = S_0; T_l = S_l diag(base phases of layer l)
        std::copy(segs[0].begin(), segs[0].end(), B.T.begin());
        for (int l = 1; l <= L; ++l) {
            std::vector<cd> d(nb_, cd(1, 0));
            for (int jj : B.layers[l - 1]) {
                const CP& cp = c->cps[jj];
                const cd ph = std::polar(1.0, 0.5 * cp.theta);
                if (cp.blk_p == b) d[local_of[cp.p]] *= ph;
                if (cp.blk_q == b) d[local_of[cp.q]] *= ph;
            }
            for (int i = 0; i < nb_; ++i)
                for (int m = 0; m < nb_; ++m) B.T[l * nn + (size_t)i * nb_ + m] = segs[l][(size_t)i * nb_ + m] * d[m];
        }

        // ---- Exact: flip patterns. A gate's pattern is the set of (layer, local
        // mode) pairs whose sign it flips; a trajectory's minor in this block
        // depends only on the XOR of its flipped gates' patterns. Local gates
        // come first so that the first r_loc basis patterns span theirs.
        B.local_gates.clear();
        for (int jj = 0; jj < k; ++jj)
            if (c->cps[jj].cls == b) B.local_gates.push_back(jj);
        B.k_loc = (int)B.local_gates.size();
        std::vector<int> gates_B = B.local_gates;
        if (c->nblocks == 2) gates_B.insert(gates_B.end(), c->shared_gates.begin(), c->shared_gates.end());
        const int PW = std::max(1, (L * nb_ + 63) / 64);
        auto pattern = [&](int jj) {
            std::vector<uint64_t> v(PW, 0);
            const CP& cp = c->cps[jj];
            const int l = layer_of_cp[jj] - 1;
            if (l >= 0) {
                if (cp.blk_p == b) {
                    const int bit = l * nb_ + local_of[cp.p];
                    v[bit >> 6] ^= 1ull << (bit & 63);
                }
                if (cp.blk_q == b) {
                    const int bit = l * nb_ + local_of[cp.q];
                    v[bit >> 6] ^= 1ull << (bit & 63);
                }
            }
            return v;
        };
        struct EchelonRow {
            std::vector<uint64_t> vec;
            uint32_t comb;
            int piv;
        };
        std::vector<EchelonRow> ech;
        std::vector<std::vector<uint64_t>> basis;
        std::vector<uint32_t> coord(gates_B.size(), 0);
        bool too_many = false;
        B.r_loc = 0;
        for (size_t gi = 0; gi < gates_B.size(); ++gi) {
            std::vector<uint64_t> v = pattern(gates_B[gi]);
            uint32_t acc = 0;
            for (const EchelonRow& e : ech)
                if ((v[e.piv >> 6] >> (e.piv & 63)) & 1ull) {
                    for (int w = 0; w < PW; ++w) v[w] ^= e.vec[w];
                    acc ^= e.comb;
                }
            int piv = -1;
            for (int w = 0; w < PW && piv < 0; ++w)
                if (v[w]) piv = w * 64 + __builtin_ctzll(v[w]);
            if (piv >= 0) {
                const int t = (int)basis.size();
                if (t >= ef::kMaxExactPatternBits) {
                    too_many = true;
                    break;
                }
                basis.push_back(pattern(gates_B[gi]));
                ech.push_back({v, acc ^ (1u << t), piv});
                coord[gi] = 1u << t;
            } else {
                coord[gi] = acc;
            }
            if ((int)gi + 1 == B.k_loc) B.r_loc = (int)basis.size();
        }
        B.r = (int)basis.size();
        B.coord = coord;
        B.local_of = local_of;
        // Gates whose flips only change signs of this block's minors: at the
        // first layer, flips of rows of S_0[:, C] that leave the support of every
        // column wholly flipped or wholly not (one sign per column); at the last
        // layer, flips of columns of S_L that do the same for every row (one sign
        // per row of the minor). Minors of patterns that differ by such gates
        // are one FP32 computation up to sign, so their rounding errors add
        // coherently: over the 2^r_sign patterns these gates span (r_sign the
        // rank of their patterns) by at most 2^(r_sign / 2) times the estimate's
        // independent sum (Cauchy-Schwarz), which fp32_err_coef applies.
        {
            const cd* S0 = &B.S[0];
            const cd* SL = &B.S[(size_t)L * nn];
            std::vector<char> fl((size_t)nb_);
            auto sign_only = [&](int jj) {
                const CP& cp = c->cps[jj];
                const int l = layer_of_cp[jj] - 1;
                std::fill(fl.begin(), fl.end(), 0);
                bool any = false;
                if (cp.blk_p == b) fl[local_of[cp.p]] ^= 1, any = true;
                if (cp.blk_q == b) fl[local_of[cp.q]] ^= 1, any = true;
                if (l < 0 || !any) return false;
                bool first_ok = l == 0, last_ok = l == L - 1;
                for (int cc = 0; first_ok && cc < B.eta; ++cc) {
                    bool f = false, u = false;
                    for (int i = 0; i < nb_; ++i)
                        if (S0[(size_t)i * nb_ + B.cols[cc]] != cd(0, 0)) (fl[i] ? f : u) = true;
                    first_ok = !(f && u);
                }
                for (int i = 0; last_ok && i < nb_; ++i) {
                    bool f = false, u = false;
                    for (int m = 0; m < nb_; ++m)
                        if (SL[(size_t)i * nb_ + m] != cd(0, 0)) (fl[m] ? f : u) = true;
                    last_ok = !(f && u);
                }
                return first_ok || last_ok;
            };
            std::vector<std::vector<uint64_t>> sech;  // echelon of the sign-only patterns
            std::vector<int> spiv;
            for (int jj : gates_B) {
                if (!sign_only(jj)) continue;
                std::vector<uint64_t> v = pattern(jj);
                for (size_t e = 0; e < sech.size(); ++e)
                    if ((v[spiv[e] >> 6] >> (spiv[e] & 63)) & 1ull)
                        for (int w = 0; w < PW; ++w) v[w] ^= sech[e][w];
                int piv = -1;
                for (int w = 0; w < PW && piv < 0; ++w)
                    if (v[w]) piv = w * 64 + __builtin_ctzll(v[w]);
                if (piv >= 0) {
                    sech.push_back(v);
                    spiv.push_back(piv);
                }
            }
            B.r_sign = (int)sech.size();
        }
        if (too_many || B.k_loc > ef::kMaxExactLocalBits || (c->nblocks == 2 && k_sh > ef::kMaxExactSharedBits)) {
            c->exact_ok = false;
            c->exact_why = "Exact mode: a mode block needs more than 2^" + std::to_string(ef::kMaxExactPatternBits) +
                           " flip patterns, more than " + std::to_string(ef::kMaxExactLocalBits) +
                           " local or more than " + std::to_string(ef::kMaxExactSharedBits) +
                           " shared controlled-phase gates";
        }
        if (B.eta > ef::kMaxEtaRows) {
            c->exact_ok = false;
            c->exact_why = "Exact mode: more than 32 particles in one mode block";
        }
        B.F.assign((size_t)L * nb_, 0u);
        for (int t = 0; t < B.r; ++t)
            for (int bit = 0; bit < L * nb_; ++bit)
                if ((basis[t][bit >> 6] >> (bit & 63)) & 1ull) B.F[bit] |= 1u << t;
        B.Omega.clear();
        B.Omega32.clear();
        B.OmegaHat.clear();
        B.OmegaHatFF.clear();
        B.sh.clear();
        B.perm.clear();
        B.goff.clear();
        B.inv_off.clear();
        B.inv_xs.clear();
        if (c->exact_ok) {
            // Omega(z) = sum of w_loc(y) over the local bit vectors y with pattern z
            static const cd ipow[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
            B.Omega.assign((size_t)1 << B.r_loc, cd(0, 0));
            const uint64_t nyl = 1ull << B.k_loc;
            for (uint64_t y = 0; y < nyl; ++y) {
                uint32_t z = 0;
                double w = 1.0;
                for (int i = 0; i < B.k_loc; ++i) {
                    const CP& cp = c->cps[B.local_gates[i]];
                    if ((y >> i) & 1ull) {
                        z ^= coord[i];
                        w *= cp.s;
                    } else {
                        w *= cp.c;
                    }
                }
                B.Omega[z] += w * ipow[__builtin_popcountll(y) & 3];
            }
            B.Omega32.resize(B.Omega.size());
            for (size_t z = 0; z < B.Omega.size(); ++z)
                B.Omega32[z] = make_float2((float)B.Omega[z].real(), (float)B.Omega[z].imag());
            // OmegaHat(u) = 2^-r_loc sum_l (-1)^{popcount(u & l)} Omega(l), by butterflies
            B.OmegaHat = B.Omega;
            for (size_t h = 1; h < B.OmegaHat.size(); h <<= 1)
                for (size_t i = 0; i < B.OmegaHat.size(); ++i)
                    if (!(i & h)) {
                        const cd a = B.OmegaHat[i], b2 = B.OmegaHat[i | h];
                        B.OmegaHat[i] = a + b2;
                        B.OmegaHat[i | h] = a - b2;
                    }
            for (cd& v : B.OmegaHat) v = std::ldexp(1.0, -B.r_loc) * v;
            B.OmegaHatFF = to_ff(B.OmegaHat);
            const int ksh_b = c->nblocks == 2 ? k_sh : 0;
            B.sh.assign((size_t)1 << ksh_b, 0u);
            for (uint32_t xs = 0; xs < (1u << ksh_b); ++xs) {
                uint32_t z = 0;
                for (int i = 0; i < ksh_b; ++i)
                    if ((xs >> i) & 1u) z ^= coord[B.k_loc + i];
                B.sh[xs] = z;
            }
            const uint32_t ngroups = 1u << (B.r - B.r_loc);
            B.goff.assign(ngroups + 1, 0u);
            for (uint32_t xs = 0; xs < B.sh.size(); ++xs) B.goff[(B.sh[xs] >> B.r_loc) + 1]++;
            for (uint32_t g = 0; g < ngroups; ++g) B.goff[g + 1] += B.goff[g];
            B.perm.assign(B.sh.size(), 0u);
            std::vector<uint32_t> fill(B.goff.begin(), B.goff.end() - 1);
            for (uint32_t xs = 0; xs < B.sh.size(); ++xs) B.perm[fill[B.sh[xs] >> B.r_loc]++] = xs;
            B.inv_off.assign(((size_t)1 << B.r) + 1, 0u);
            for (uint32_t xs = 0; xs < B.sh.size(); ++xs) B.inv_off[B.sh[xs] + 1]++;
            for (size_t z = 0; z + 1 < B.inv_off.size(); ++z) B.inv_off[z + 1] += B.inv_off[z];
            B.inv_xs.assign(B.sh.size(), 0u);
            std::vector<uint32_t> fz(B.inv_off.begin(), B.inv_off.end() - 1);
            for (uint32_t xs = 0; xs < B.sh.size(); ++xs) B.inv_xs[fz[B.sh[xs]]++] = xs;
        }

        // ---- Raw Estimate: interval products and right factors
        B.P.assign((size_t)(tri(L, L) + 1) * nn, cd(0, 0));
        for (int bb = 0; bb <= L; ++bb) {
            // Pi_{bb..bb} = T_bb; Pi_{a..bb} = T_a Pi_{a-1..bb}
            std::copy(B.T.begin() + bb * nn, B.T.begin() + (bb + 1) * nn, B.P.begin() + (size_t)tri(bb, bb) * nn);
            for (int a = bb + 1; a <= L; ++a) {
                const cd* Ta = &B.T[a * nn];
                const cd* prev = &B.P[(size_t)tri(a - 1, bb) * nn];
                cd* out = &B.P[(size_t)tri(a, bb) * nn];
                for (int i = 0; i < nb_; ++i)
                    for (int jj = 0; jj < nb_; ++jj) {
                        cd acc = 0;
                        for (int m = 0; m < nb_; ++m) acc += Ta[(size_t)i * nb_ + m] * prev[(size_t)m * nb_ + jj];
                        out[(size_t)i * nb_ + jj] = acc;
                    }
            }
        }
        B.RC.assign((size_t)L * nb_ * B.eta, cd(0, 0));
        for (int l = 0; l < L; ++l) {
            const cd* Pl0 = &B.P[(size_t)tri(l, 0) * nn];
            for (int i = 0; i < nb_; ++i)
                for (int cc = 0; cc < B.eta; ++cc)
                    B.RC[((size_t)l * nb_ + i) * B.eta + cc] = Pl0[(size_t)i * nb_ + B.cols[cc]];
        }
        if (B.eta > ef::kMaxApproxEta) {
            c->approx_ok = false;
            c->approx_why = "Raw Estimate: more than 13 particles in one mode block";
        }
        if (L > ef::kMaxApproxLayers || nb_ > 64 || (L > 0 && (L - 1) * nb_ > ef::kMaxApproxStored)) {
            c->approx_ok = false;
            c->approx_why = "Raw Estimate: mode block with more than 64 modes, more than 8 controlled-phase "
                            "layers, or (layers-1)*modes above 64";
        }
        for (int jj = 0; jj < k; ++jj) {
            const CP& cp = c->cps[jj];
            uint64_t mm = 0;
            if (cp.blk_p == b) mm ^= 1ull << local_of[cp.p];
            if (cp.blk_q == b) mm ^= 1ull << local_of[cp.q];
            c->alayer[(size_t)b * k + jj] = (uint8_t)((cp.blk_p == b || cp.blk_q == b) ? layer_of_cp[jj] : 0);
            c->amodes[(size_t)b * k + jj] = (nb_ <= 64) ? mm : 0;
        }
        // Raw Estimate K form: the (layer, mode) pairs some gate can flip, layer-major
        B.pair_lm.clear();
        if (nb_ <= 64) {
            std::vector<std::vector<int>> pidx(L + 1, std::vector<int>(nb_, -1));
            for (int l = 1; l <= L; ++l) {
                uint64_t any = 0;
                for (int jj = 0; jj < k; ++jj)
                    if (c->alayer[(size_t)b * k + jj] == l) any |= c->amodes[(size_t)b * k + jj];
                for (int m = 0; m < nb_; ++m)
                    if ((any >> m) & 1ull) {
                        pidx[l][m] = (int)B.pair_lm.size();
                        B.pair_lm.push_back((l << 8) | m);
                    }
            }
            if (B.pair_lm.size() > 64) {
                c->kform_ok = false;
            } else {
                for (int jj = 0; jj < k; ++jj) {
                    const int l = c->alayer[(size_t)b * k + jj];
                    uint64_t mm = c->amodes[(size_t)b * k + jj], g = 0;
                    while (l && mm) {
                        const int m = __builtin_ctzll(mm);
                        mm &= mm - 1;
                        g ^= 1ull << pidx[l][m];
                    }
                    c->agpair[(size_t)b * k + jj] = g;
                }
            }
        } else {
            c->kform_ok = false;
        }
    }
    // shared weight table: w_sh(x_sh) = i^|x_sh| prod_j (x_j ? s_j : c_j)
    c->WS.clear();
    if (c->exact_ok) {
        const int ksh_b = c->nblocks == 2 ? k_sh : 0;
        c->WS.assign((size_t)1 << ksh_b, cd(0, 0));
        static const cd ipow[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
        for (uint32_t xs = 0; xs < (1u << ksh_b); ++xs) {
            double w = 1.0;
            for (int i = 0; i < ksh_b; ++i) {
                const CP& cp = c->cps[c->shared_gates[i]];
                w *= ((xs >> i) & 1u) ? cp.s : cp.c;
            }
            c->WS[xs] = w * ipow[__builtin_popcount(xs) & 3];
        }
        c->WS32.resize(c->WS.size());
        for (size_t x = 0; x < c->WS.size(); ++x)
            c->WS32[x] = make_float2((float)c->WS[x].real(), (float)c->WS[x].imag());
        c->WSFF = to_ff(c->WS);
    }
    c->p_floor = 1e-6 * std::exp(-log_sector);
    // approx gate tables
    c->aT.assign(k, 0);
    c->aq.assign(k, 0.0);
    c->aq32.assign(k, 0.f);
    c->R0 = 1.0;
    for (int jj = 0; jj < k; ++jj) {
        const CP& cp = c->cps[jj];
        c->aT[jj] = cp.T;
        c->aq[jj] = cp.ratio0 != 0.0 ? cp.ratio1 / cp.ratio0 : 0.0;
        c->aq32[jj] = (float)c->aq[jj];
        c->R0 *= cp.ratio0;
    }
    c->dirty = true;
    ++c->tables_gen;
    return EF_OK;
}

std::vector<double2> to_d2(const std::vector<cd>& v, size_t off = 0, size_t count = (size_t)-1) {
    const size_t n = std::min(count, v.size() - std::min(off, v.size()));
    std::vector<double2> o(n);
    for (size_t i = 0; i < n; ++i) o[i] = make_double2(v[off + i].real(), v[off + i].imag());
    return o;
}

int upload_tables(ef_circuit* c, cudaStream_t s) {
    if (!c->dirty) return EF_OK;
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const size_t nn = (size_t)B.n * B.n;
        std::vector<double2> S0C((size_t)B.n * B.eta);
        for (int i = 0; i < B.n; ++i)
            for (int cc = 0; cc < B.eta; ++cc) {
                const cd v = B.S[(size_t)i * B.n + B.cols[cc]];
                S0C[(size_t)i * B.eta + cc] = make_double2(v.real(), v.imag());
            }
        EF_CK(upload(B.dS0C, S0C, s));
        EF_CK(upload(B.dT, to_d2(B.T, nn, (size_t)B.L * nn), s));
        EF_CK(upload(B.dF, B.F, s));
        EF_CK(upload(B.dOmega, to_d2(B.Omega), s));
        EF_CK(upload(B.dOmega32, B.Omega32, s));
        EF_CK(upload(B.dOmegaHat, to_d2(B.OmegaHat), s));
        EF_CK(upload(B.dOmegaHatFF, B.OmegaHatFF, s));
        EF_CK(upload(B.dSh, B.sh, s));
        EF_CK(upload(B.dPerm, B.perm, s));
        EF_CK(upload(B.dGoff, B.goff, s));
        EF_CK(upload(B.dInvOff, B.inv_off, s));
        EF_CK(upload(B.dInvXs, B.inv_xs, s));
        std::vector<float2> P32(B.P.size()), RC32(B.RC.size());
        for (size_t e = 0; e < B.P.size(); ++e) P32[e] = make_float2((float)B.P[e].real(), (float)B.P[e].imag());
        for (size_t e = 0; e < B.RC.size(); ++e) RC32[e] = make_float2((float)B.RC[e].real(), (float)B.RC[e].imag());
        EF_CK(upload(B.dP64, to_d2(B.P), s));
        EF_CK(upload(B.dP32, P32, s));
        EF_CK(upload(B.dRC64, to_d2(B.RC), s));
        EF_CK(upload(B.dRC32, RC32, s));
        EF_CK(upload(B.dCols, B.cols, s));
        EF_CK(upload(B.dPairLM, B.pair_lm, s));
    }
    EF_CK(upload(c->dWS, to_d2(c->WS), s));
    EF_CK(upload(c->dWS32, c->WS32, s));
    EF_CK(upload(c->dWSFF, c->WSFF, s));
    std::vector<uint32_t> T4(((c->aT.size() + 3) & ~(size_t)3), 0u);
    std::copy(c->aT.begin(), c->aT.end(), T4.begin());
    EF_CK(upload(c->daT, T4, s));
    EF_CK(upload(c->daq, c->aq, s));
    EF_CK(upload(c->daq32, c->aq32, s));
    EF_CK(upload(c->dalayer, c->alayer, s));
    EF_CK(upload(c->damodes, c->amodes, s));
    EF_CK(upload(c->dagpair, c->agpair, s));
    c->dirty = false;
    return EF_OK;
}

int validate_gates(int n, const ef_gate* gates, int64_t ng) {
    for (int64_t i = 0; i < ng; ++i) {
        const ef_gate& g = gates[i];
        const std::string at = "gate " + std::to_string(i) + ": ";
        if (g.reserved != 0) return fail(EF_EINVAL, at + "reserved field must be 0");
        if (g.p < 0 || g.p >= n) return fail(EF_EINVAL, at + "mode p out of range");
        switch (g.kind) {
            case EF_GIVENS:
                if (g.q != g.p + 1 || g.q >= n)
                    return fail(EF_EINVAL, at + "Givens rotations act on adjacent modes (q = p + 1 < n)");
                if (!std::isfinite(g.theta) || !std::isfinite(g.phi)) return fail(EF_EINVAL, at + "non-finite angle");
                break;
            case EF_PHASE:
                if (!std::isfinite(g.phi)) return fail(EF_EINVAL, at + "non-finite angle");
                break;
            case EF_CPHASE:
                if (g.q < 0 || g.q >= n || g.q == g.p) return fail(EF_EINVAL, at + "controlled phase needs p != q < n");
                if (!std::isfinite(g.theta)) return fail(EF_EINVAL, at + "non-finite angle");
                break;
            default:
                return fail(EF_EINVAL, at + "unknown gate kind");
        }
    }
    return EF_OK;
}

double lu_flops(int eta) {
    double f = 17.0 * eta;
    for (int k = 0; k < eta; ++k) {
        const double r = eta - k - 1;
        f += 8.0 * r * r + 6.0 * r;
    }
    return f;
}

int begin_call(ef_circuit* c, cudaStream_t s, int mode) {
    if (c->has_last_stream && c->last_stream != s) EF_CK(cudaStreamSynchronize(c->last_stream));
    c->last_stream = s;
    c->has_last_stream = true;
    c->stats = ef_stats{};
    c->last_mode = mode;
    c->last_fp64_list_pending = 0;
    c->last_recomp = nullptr;
    c->timed = (c->opt.flags & EF_FLAG_TIME_KERNELS) != 0;
    if (c->timed && !c->ev0) {
        EF_CK(cudaEventCreate(&c->ev0));
        EF_CK(cudaEventCreate(&c->ev1));
    }
    return upload_tables(c, s);
}

// Device buffers of one Exact call (from the circuit's workspace or from the
// allocation-free scratch).
struct ExactBuffers {
    ef::ExactBlockDev blk[ef::kMaxBlocks];
    const double2* Omega[ef::kMaxBlocks];
    const float2* Omega32[ef::kMaxBlocks];
    const double2* OmegaHat[ef::kMaxBlocks];
    const float4* OmegaHatFF[ef::kMaxBlocks];
    const uint32_t* sh[ef::kMaxBlocks];
    const uint32_t* perm[ef::kMaxBlocks];
    const uint32_t* goff[ef::kMaxBlocks];
    const uint32_t* inv_off[ef::kMaxBlocks];
    const uint32_t* inv_xs[ef::kMaxBlocks];
    const double2* WS;
    const float2* WS32;
    const float4* WSFF;
    int* list;   // bitstrings flagged by the FP32 pass
    int* list2;  // bitstrings still above tol after their listed determinants were redone
    int* count;  // [0] list size, [1] list2 size, [2 + B] listed determinants of block B
    int2* mlist[ef::kMaxBlocks];  // (column, pattern) of the determinants to redo in FP64
    unsigned long long* recomp;   // [0] bitstrings, [1] determinants recomputed in FP64
    int64_t cap;  // bitstrings per batch (row stride of the determinant buffers)
};

// EF_PREC_AUTO redoes single determinants (rather than whole bitstrings) when
// the thread-per-minor FP64 kernel covers every block and the combine can hold
// one variance term per determinant in shared memory.
bool per_minor_recompute(const ef_circuit* c) {
    if (c->opt.precision != EF_PREC_AUTO || c->nblocks == 0) return false;
    int64_t minors = 0;
    for (int b = 0; b < c->nblocks; ++b) {
        if (c->blk[b].eta > 8) return false;
        minors += (int64_t)1 << c->blk[b].r;
    }
    return minors <= 8192;
}

// Bytes per (pattern, bitstring) determinant: FP32 results (float2 value and
// a 16-bit error term) unless FP64-only, FP64 ones (double2) for FP64 and for
// the recomputes of AUTO.
size_t det_bytes(const ef_circuit* c) {
    const int p = c->opt.precision;
    return (p != EF_PREC_FP64 ? sizeof(float2) + sizeof(uint16_t) : 0) +
           (p != EF_PREC_FP32_MINOR ? sizeof(double2) : 0);
}

// Bitstrings per batch so that the per-(pattern, bitstring) determinants stay
// within `budget` bytes.
int64_t exact_batch(const ef_circuit* c, int64_t nb, size_t budget) {
    size_t per = 0;
    const size_t each = det_bytes(c) + (per_minor_recompute(c) ? sizeof(int2) : 0);
    for (int b = 0; b < c->nblocks; ++b) per += ((size_t)1 << c->blk[b].r) * each;
    if (per == 0 || nb == 0) return std::max<int64_t>(nb, 1);
    return std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)(budget / per)));
}

void exact_block_geometry(const ef_circuit* c, int b, int64_t cap, ef::ExactBlockDev& d) {
    const HostBlock& B = c->blk[b];
    d.n = B.n;
    d.eta = B.eta;
    d.L = B.L;
    d.r = B.r;
    d.r_loc = B.r_loc;
    // ef_options.tile_override[0] > 0 fixes the patterns per chunk (log2), within the
    // pattern count and 96 KiB of staged matrices
    int cl = c->opt.tile_override[0];
    if (cl > 0) {
        cl = std::min(cl, B.r);
        while (cl > 0 && ((size_t)1 << cl) * B.n * (size_t)(B.eta | 1) * sizeof(float2) > 96 * 1024) --cl;
    } else {
        cl = ef::exact_f32_chunk_log2(B.n, B.eta, B.r, cap);
    }
    d.c_log2 = cl;
    d.n_chunks = 1 << (B.r - d.c_log2);
    d.mask0 = B.mask[0];
    d.mask1 = B.mask[1];
}

// The transform path of the combine holds both blocks' 2^r values in shared
// memory (at most 64 KiB) and pays off once the direct sums' 2^(k_sh + r_loc)
// complex multiply-adds per block exceed the transforms' work.
bool combine_by_transforms(const ef_circuit* c) {
    if (c->nblocks != 2) return false;
    double direct = 0.0, wht = 0.0;
    for (int b = 0; b < 2; ++b) {
        const HostBlock& B = c->blk[b];
        if (B.r_loc < 1 || B.r > 11) return false;
        direct += 4.0 * std::ldexp(1.0, (int)c->shared_gates.size() + B.r_loc);
        wht += std::ldexp(1.0, B.r) * (4.0 * B.r_loc + 4.0);
    }
    return wht < direct;
}

ef::ExactCombineDev make_combine(const ef_circuit* c, const ExactBuffers& eb) {
    ef::ExactCombineDev cm{};
    cm.nblocks = c->nblocks;
    cm.k_sh = c->nblocks == 2 ? (int)c->shared_gates.size() : 0;
    cm.inactive0 = c->inactive[0];
    cm.inactive1 = c->inactive[1];
    for (int b = 0; b < c->nblocks; ++b) {
        cm.mask[b][0] = c->blk[b].mask[0];
        cm.mask[b][1] = c->blk[b].mask[1];
        cm.eta[b] = c->blk[b].eta;
        cm.r[b] = c->blk[b].r;
        cm.r_loc[b] = c->blk[b].r_loc;
        cm.D32[b] = eb.blk[b].D32;
        cm.E32[b] = eb.blk[b].E32;
        cm.D64[b] = eb.blk[b].D64;
        cm.OmegaHatDF[b] = eb.OmegaHatFF[b];
        cm.Omega[b] = eb.Omega[b];
        cm.Omega32[b] = eb.Omega32[b];
        cm.OmegaHat[b] = eb.OmegaHat[b];
        cm.s[b] = eb.sh[b];
        cm.perm[b] = eb.perm[b];
        cm.goff[b] = eb.goff[b];
        cm.inv_off[b] = eb.inv_off[b];
        cm.inv_xs[b] = eb.inv_xs[b];
    }
    cm.WS = eb.WS;
    cm.WS32 = eb.WS32;
    cm.WSDF = eb.WSFF;
    cm.src = c->opt.precision == EF_PREC_FP64 ? 1 : 0;
    cm.wht = combine_by_transforms(c) ? 1 : 0;
    cm.inj = c->nblocks == 2 ? 1 : 0;
    for (int b = 0; b < c->nblocks && cm.inj; ++b)
        for (size_t z = 0; z + 1 < c->blk[b].inv_off.size(); ++z)
            if (c->blk[b].inv_off[z + 1] - c->blk[b].inv_off[z] > 1) cm.inj = 0;
    cm.wreg = 0;
    if (cm.wht && c->opt.precision != EF_PREC_FP64) {
        cm.wreg = 1;
        for (int b = 0; b < 2; ++b)
            if (c->blk[b].r < 5 || c->blk[b].r > 10 || c->blk[b].r_loc > 5) cm.wreg = 0;
    }
    cm.minors = 0;
    for (int b = 0; b < c->nblocks; ++b) cm.minors += (int64_t)1 << c->blk[b].r;
    cm.mcount = eb.count + 2;
    cm.tol = c->opt.tol;
    cm.p_floor = c->p_floor;
    return cm;
}

// FP32 error model: per minor |d det|^2 ~ (K u32)^2 (|det|^2 er2 + zabs2),
// independent between distinct minors and propagated to the amplitude
// through each minor's coefficient. Observed errors behave like Gaussians
// whose standard deviation is about a third of the K = 1 estimate, so K = 4
// bounds them at about 5 standard deviations (the largest ratio seen in
// 16,000 significant results was 0.76 at K = 4); ef_options.tile_override[1]
// > 0 sets K in tenths. Minors that are one computation up to sign are not
// independent: for a block with r_sign such pattern directions the coefficient
// takes a factor 2^(r_sign / 2) (one for circuits whose controlled-phase gates
// all sit between rotations).
double fp32_err_coef(const ef_circuit* c) {
    if (c->opt.precision == EF_PREC_FP64) return 0.0;
    const double K = c->opt.tile_override[1] > 0 ? 0.1 * c->opt.tile_override[1] : 4.0;
    int rs = 0;  // coherent rounding errors of minors equal up to sign (HostBlock::r_sign)
    for (int b = 0; b < c->nblocks; ++b) rs = std::max(rs, c->blk[b].r_sign);
    return K * std::ldexp(1.0, -24) * std::sqrt(std::ldexp(1.0, rs));
}

void exact_account(ef_circuit* c, int64_t nb) {
    double flops = 0.0;
    int64_t sub_total = 0;
    for (int b = 0; b < c->nblocks; ++b) {
        flops += (double)nb * std::ldexp(1.0, c->blk[b].r) * lu_flops(c->blk[b].eta);
        sub_total += (int64_t)1 << c->blk[b].r;
    }
    c->last_sub_total = sub_total;
    c->stats.dominant_kernel_flops = flops;
}

int exact_enqueue_build(ef_circuit* c, const ExactBuffers& eb, cudaStream_t s, ef::LaunchStats& st) {
    const bool fp64_only = c->opt.precision == EF_PREC_FP64;
    if (c->nblocks > 0) EF_CK(ef::launch_build_branches(eb.blk[0], eb.blk[1], c->nblocks, !fp64_only, s, st));
    return EF_OK;
}

int exact_enqueue_lu(ef_circuit* c, const ExactBuffers& eb, const uint64_t* bits, int64_t nbb, cudaStream_t s,
                     ef::LaunchStats& st) {
    const bool fp64_only = c->opt.precision == EF_PREC_FP64;
    if (!fp64_only && c->nblocks == 2 && eb.blk[0].eta == eb.blk[1].eta && eb.blk[0].eta <= ef::kMaxEtaThread) {
        EF_CK(ef::launch_exact_lu_f32(eb.blk[0], eb.blk[1], 2, bits, nbb, s, st));
        return EF_OK;
    }
    for (int b = 0; b < c->nblocks; ++b) {
        const ef::ExactBlockDev& d = eb.blk[b];
        if (fp64_only) {
            EF_CK(ef::launch_exact_lu_f64(d, bits, nbb, nullptr, nullptr, nbb, s, st));
        } else if (d.eta <= ef::kMaxEtaThread) {
            EF_CK(ef::launch_exact_lu_f32(d, d, 1, bits, nbb, s, st));
        } else {
            EF_CK(ef::launch_exact_lu_rows(d, bits, nbb, nullptr, nullptr, nbb, false, s, st));
        }
    }
    return EF_OK;
}

// combine, and under EF_PREC_AUTO the FP64 recompute of flagged results:
// per determinant when eb.mlist is set (FP32 pass -> listed determinants in
// FP64 -> combine of the flagged bitstrings with a new estimate -> whole
// bitstrings still above tol in FP64 -> their combine), else per bitstring.
int exact_enqueue_combine(ef_circuit* c, const ExactBuffers& eb, ef::ExactCombineDev cm, const uint64_t* bits,
                          int64_t nbb, double* out, double* err, cudaStream_t s, ef::LaunchStats& st) {
    const bool autofix = c->opt.precision == EF_PREC_AUTO;
    cm.err_coef = fp32_err_coef(c);
    if (!autofix) {
        EF_CK(ef::launch_exact_combine(cm, bits, nbb, nbb, nullptr, nullptr, out, err, nullptr, nullptr, s, st));
        return EF_OK;
    }
    const bool per_minor = eb.mlist[0] != nullptr;
    EF_CK(cudaMemsetAsync(eb.count, 0, 4 * sizeof(int), s));
    for (int b = 0; b < c->nblocks; ++b) cm.mlist[b] = per_minor ? eb.mlist[b] : nullptr;
    EF_CK(ef::launch_exact_combine(cm, bits, nbb, nbb, nullptr, nullptr, out, err, eb.list, eb.count, s, st));
    for (int b = 0; b < c->nblocks; ++b) cm.mlist[b] = nullptr;
    cm.recomp = eb.recomp;
    if (per_minor) {
        if (c->nblocks == 2 && eb.blk[0].eta == eb.blk[1].eta) {
            EF_CK(ef::launch_exact_lu_redo_minors(eb.blk[0], eb.blk[1], 2, bits, eb.mlist[0], eb.mlist[1],
                                                  eb.count + 2, s, st));
        } else {
            for (int b = 0; b < c->nblocks; ++b)
                EF_CK(ef::launch_exact_lu_redo_minors(eb.blk[b], eb.blk[b], 1, bits, eb.mlist[b], nullptr,
                                                      eb.count + 2 + b, s, st));
        }
        ef::ExactCombineDev chk = cm;
        chk.src = 2;
        chk.col_by_index = 1;
        chk.count_bits = 1;
        chk.count_minors = 1;
        EF_CK(ef::launch_exact_combine(chk, bits, nbb, nbb, eb.list, eb.count, out, err, eb.list2, eb.count + 1, s,
                                       st));
        for (int b = 0; b < c->nblocks; ++b)
            EF_CK(ef::launch_exact_lu_f64(eb.blk[b], bits, nbb, eb.list2, eb.count + 1, nbb, s, st));
        cm.err_coef = 0.0;
        cm.src = 1;
        cm.count_full = 1;
        EF_CK(ef::launch_exact_combine(cm, bits, nbb, nbb, eb.list2, eb.count + 1, out, err, nullptr, nullptr, s,
                                       st));
    } else {
        for (int b = 0; b < c->nblocks; ++b)
            EF_CK(ef::launch_exact_lu_f64(eb.blk[b], bits, nbb, eb.list, eb.count, nbb, s, st));
        cm.err_coef = 0.0;
        cm.src = 1;
        cm.count_bits = 1;
        cm.count_full = 1;
        EF_CK(ef::launch_exact_combine(cm, bits, nbb, nbb, eb.list, eb.count, out, err, nullptr, nullptr, s, st));
    }
    return EF_OK;
}

int run_exact(ef_circuit* c, const ExactBuffers& eb, const uint64_t* d_bits, int64_t nb, double* d_out,
              double* d_err, cudaStream_t s, ef::LaunchStats& st) {
    const bool autofix = c->opt.precision == EF_PREC_AUTO;
    exact_account(c, nb);
    int rc = exact_enqueue_build(c, eb, s, st);
    if (rc) return rc;
    const ef::ExactCombineDev cm = make_combine(c, eb);
    if (autofix) {
        EF_CK(cudaMemsetAsync(eb.recomp, 0, 2 * sizeof(unsigned long long), s));
        c->last_recomp = eb.recomp;
        c->last_fp64_list_pending = 1;
    }
    int64_t lu_launches = 0;
    for (int64_t off = 0; off < nb; off += eb.cap) {
        const int64_t nbb = std::min(eb.cap, nb - off);
        const uint64_t* bits = d_bits + 2 * off;
        if (c->timed && off == 0) EF_CK(cudaEventRecord(c->ev0, s));
        const int64_t before = st.launches;
        rc = exact_enqueue_lu(c, eb, bits, nbb, s, st);
        if (rc) return rc;
        lu_launches += st.launches - before;
        if (c->timed && off + nbb >= nb) EF_CK(cudaEventRecord(c->ev1, s));
        rc = exact_enqueue_combine(c, eb, cm, bits, nbb, d_out + off, d_err ? d_err + off : nullptr, s, st);
        if (rc) return rc;
    }
    c->stats.dominant_kernel_launches = lu_launches;
    c->stats.kernel_launches = st.launches;
    c->stats.executed_minor_lus = st.executed_lus;
    return EF_OK;
}

// Workspace and device pointers of an Exact call with batches of `cap` bitstrings.
int exact_buffers(ef_circuit* c, int64_t cap, ExactBuffers& eb) {
    const bool fp64_only = c->opt.precision == EF_PREC_FP64;
    eb = ExactBuffers{};
    eb.cap = cap;
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const size_t ny = (size_t)1 << B.r;
        const size_t ne = (size_t)B.n * B.eta;
        EF_CK(B.dM64.ensure(ny * ne * sizeof(double2)));
        if (!fp64_only) EF_CK(B.dM32.ensure(2 * ny * ne * sizeof(float2)));
        const bool d32 = c->opt.precision != EF_PREC_FP64, d64 = c->opt.precision != EF_PREC_FP32_MINOR;
        if (d32) EF_CK(B.dD32.ensure(ny * (size_t)cap * sizeof(float2)));
        if (d32) EF_CK(B.dE32.ensure(ny * (size_t)cap * sizeof(uint16_t)));
        if (d64) EF_CK(B.dD64.ensure(ny * (size_t)cap * sizeof(double2)));
        ef::ExactBlockDev& d = eb.blk[b];
        exact_block_geometry(c, b, cap, d);
        d.S0C = B.dS0C.as<double2>();
        d.T = B.dT.as<double2>();
        d.F = B.dF.as<uint32_t>();
        d.M64 = B.dM64.as<double2>();
        d.M32 = fp64_only ? nullptr : B.dM32.as<float2>();
        d.ML32 = fp64_only ? nullptr : B.dM32.as<float2>() + ny * ne;
        d.D32 = d32 ? B.dD32.as<float2>() : nullptr;
        d.E32 = d32 ? B.dE32.as<uint16_t>() : nullptr;
        d.D64 = d64 ? B.dD64.as<double2>() : nullptr;
        eb.Omega[b] = B.dOmega.as<double2>();
        eb.Omega32[b] = B.dOmega32.as<float2>();
        eb.OmegaHat[b] = B.dOmegaHat.as<double2>();
        eb.OmegaHatFF[b] = B.dOmegaHatFF.as<float4>();
        eb.sh[b] = B.dSh.as<uint32_t>();
        eb.perm[b] = B.dPerm.as<uint32_t>();
        eb.goff[b] = B.dGoff.as<uint32_t>();
        eb.inv_off[b] = B.dInvOff.as<uint32_t>();
        eb.inv_xs[b] = B.dInvXs.as<uint32_t>();
    }
    eb.WS = c->dWS.as<double2>();
    eb.WS32 = c->dWS32.as<float2>();
    eb.WSFF = c->dWSFF.as<float4>();
    EF_CK(c->dList.ensure(2 * (size_t)cap * sizeof(int)));
    EF_CK(c->dListCount.ensure(4 * sizeof(int)));
    EF_CK(c->dRecomp.ensure(2 * sizeof(unsigned long long)));
    eb.list = c->dList.as<int>();
    eb.list2 = eb.list + cap;
    eb.count = c->dListCount.as<int>();
    eb.recomp = c->dRecomp.as<unsigned long long>();
    if (per_minor_recompute(c))
        for (int b = 0; b < c->nblocks; ++b) {
            HostBlock& B = c->blk[b];
            EF_CK(B.dMlist.ensure(((size_t)1 << B.r) * (size_t)cap * sizeof(int2)));
            eb.mlist[b] = B.dMlist.as<int2>();
        }
    return EF_OK;
}

int exact_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, double* d_out, double* d_err, cudaStream_t s) {
    if (!c->exact_ok) return fail(EF_EUNSUPPORTED, c->exact_why);
    int rc = begin_call(c, s, 1);
    if (rc) return rc;
    c->stats.logical_branch_dets = nb * (int64_t)std::ldexp(1.0, (int)c->cps.size());
    if (nb == 0) return EF_OK;
    ExactBuffers eb;
    rc = exact_buffers(c, exact_batch(c, nb, (size_t)2 << 30), eb);
    if (rc) return rc;
    ef::LaunchStats st;
    return run_exact(c, eb, d_bits, nb, d_out, d_err, s, st);
}

// ------------------------------------------------------------------ adjoint (host part)

// Chain rule from the device cotangents to the angle vector.
//   tbar[b][l]: d L / d T_{l+1} (n x n), sbar[b]: d L / d S_0[:, C] (n x eta),
//   ebar[b]: d L / d Omega_b(z_local), pbar: d L / d w_sh(x_sh); all bilinear
//   (dL = Re sum cot * d value).
void grad_finish(const ef_circuit* c, const std::vector<std::vector<cd>>& tbar, const std::vector<std::vector<cd>>& sbar,
                 const std::vector<std::vector<cd>>& ebar, const std::vector<cd>& pbar, std::vector<double>& grad) {
    const cd I(0.0, 1.0);
    static const cd ipow[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
    std::vector<int64_t> aidx(c->gates.size());
    int64_t na = 0;
    for (size_t gi = 0; gi < c->gates.size(); ++gi) {
        aidx[gi] = na;
        na += c->gates[gi].kind == EF_GIVENS ? 2 : 1;
    }
    grad.assign(na, 0.0);
    // weights: w(y) = i^|y| prod_t (y_t ? s_t : c_t), ds/dtheta = c/4, dc/dtheta = -s/4
    auto weight_grads = [&](const std::vector<int>& gates, const std::vector<uint32_t>& coord, int coff,
                            const std::vector<cd>& cot, bool by_pattern) {
        const int kk = (int)gates.size();
        if (kk == 0) return;
        std::vector<double> pre(kk + 1), suf(kk + 1);
        for (uint64_t y = 0; y < (1ull << kk); ++y) {
            uint32_t z = 0;
            pre[0] = 1.0;
            for (int t = 0; t < kk; ++t) {
                const CP& cp = c->cps[gates[t]];
                const bool bit = (y >> t) & 1ull;
                if (bit && by_pattern) z ^= coord[coff + t];
                pre[t + 1] = pre[t] * (bit ? cp.s : cp.c);
            }
            suf[kk] = 1.0;
            for (int t = kk - 1; t >= 0; --t) {
                const CP& cp = c->cps[gates[t]];
                suf[t] = suf[t + 1] * (((y >> t) & 1ull) ? cp.s : cp.c);
            }
            const cd e = cot[by_pattern ? z : (uint32_t)y] * ipow[__builtin_popcountll(y) & 3];
            for (int t = 0; t < kk; ++t) {
                const CP& cp = c->cps[gates[t]];
                const double dfac = ((y >> t) & 1ull) ? 0.25 * cp.c : -0.25 * cp.s;
                grad[aidx[cp.gate]] += (e * (pre[t] * suf[t + 1] * dfac)).real();
            }
        }
    };
    for (int b = 0; b < c->nblocks; ++b) weight_grads(c->blk[b].local_gates, c->blk[b].coord, 0, ebar[b], true);
    if (c->nblocks == 2) weight_grads(c->shared_gates, {}, 0, pbar, false);

    for (int b = 0; b < c->nblocks; ++b) {
        const HostBlock& B = c->blk[b];
        const int n = B.n;
        const size_t nn = (size_t)n * n;
        std::vector<std::vector<cd>> Sbar(B.L + 1, std::vector<cd>(nn, cd(0, 0)));
        for (int i = 0; i < n; ++i)
            for (int cc = 0; cc < B.eta; ++cc) Sbar[0][(size_t)i * n + B.cols[cc]] = sbar[b][(size_t)i * B.eta + cc];
        for (int l = 1; l <= B.L; ++l) {
            std::vector<cd> d(n, cd(1, 0));
            for (int jj : B.layers[l - 1]) {
                const CP& cp = c->cps[jj];
                const cd ph = std::polar(1.0, 0.5 * cp.theta);
                if (cp.blk_p == b) d[B.local_of[cp.p]] *= ph;
                if (cp.blk_q == b) d[B.local_of[cp.q]] *= ph;
            }
            const cd* Tb = &tbar[b][(size_t)(l - 1) * nn];
            const cd* S = &B.S[(size_t)l * nn];
            std::vector<cd> dbar(n, cd(0, 0));
            for (int i = 0; i < n; ++i)
                for (int m = 0; m < n; ++m) {
                    dbar[m] += Tb[(size_t)i * n + m] * S[(size_t)i * n + m];
                    Sbar[l][(size_t)i * n + m] = Tb[(size_t)i * n + m] * d[m];
                }
            for (int jj : B.layers[l - 1]) {
                const CP& cp = c->cps[jj];
                for (int side = 0; side < 2; ++side) {
                    const int mode = side ? cp.q : cp.p;
                    if ((side ? cp.blk_q : cp.blk_p) != b) continue;
                    const int m = B.local_of[mode];
                    grad[aidx[cp.gate]] += (dbar[m] * (0.5 * I) * d[m]).real();
                }
            }
        }
        // segments S_l = G_K ... G_1: dL/dG_k = (G_K..G_{k+1})^T Sbar (G_{k-1}..G_1)^T
        for (int l = 0; l <= B.L; ++l) {
            std::vector<cd> M = Sbar[l];
            std::vector<cd> R(B.S.begin() + (size_t)l * nn, B.S.begin() + (size_t)(l + 1) * nn);
            const std::vector<int>& seq = B.seg_gates[l];
            for (int kk = (int)seq.size() - 1; kk >= 0; --kk) {
                const ef_gate& g = c->gates[seq[kk]];
                const int lp = B.local_of[g.p];
                if (g.kind == EF_GIVENS) {
                    const int lq = B.local_of[g.q];
                    const double ct = std::cos(g.theta), st = std::sin(g.theta);
                    const cd e = std::polar(1.0, g.phi), em = std::polar(1.0, -g.phi);
                    const cd G[2][2] = {{ct, -e * st}, {em * st, ct}};
                    const cd dT[2][2] = {{-st, -e * ct}, {em * ct, -st}};
                    const cd dP[2][2] = {{0.0, -I * e * st}, {-I * em * st, 0.0}};
                    for (int col = 0; col < n; ++col) {
                        const cd a = R[(size_t)lp * n + col], bb = R[(size_t)lq * n + col];
                        R[(size_t)lp * n + col] = std::conj(G[0][0]) * a + std::conj(G[1][0]) * bb;
                        R[(size_t)lq * n + col] = std::conj(G[0][1]) * a + std::conj(G[1][1]) * bb;
                    }
                    const int ix[2] = {lp, lq};
                    cd Gb[2][2];
                    for (int a = 0; a < 2; ++a)
                        for (int bb = 0; bb < 2; ++bb) {
                            cd acc = 0;
                            for (int col = 0; col < n; ++col) acc += M[(size_t)ix[a] * n + col] * R[(size_t)ix[bb] * n + col];
                            Gb[a][bb] = acc;
                        }
                    double gt = 0.0, gp = 0.0;
                    for (int a = 0; a < 2; ++a)
                        for (int bb = 0; bb < 2; ++bb) {
                            gt += (Gb[a][bb] * dT[a][bb]).real();
                            gp += (Gb[a][bb] * dP[a][bb]).real();
                        }
                    grad[aidx[seq[kk]]] += gt;
                    grad[aidx[seq[kk]] + 1] += gp;
                    for (int col = 0; col < n; ++col) {
                        const cd a = M[(size_t)lp * n + col], bb = M[(size_t)lq * n + col];
                        M[(size_t)lp * n + col] = G[0][0] * a + G[1][0] * bb;
                        M[(size_t)lq * n + col] = G[0][1] * a + G[1][1] * bb;
                    }
                } else {  // PHASE
                    const cd e = std::polar(1.0, g.phi);
                    for (int col = 0; col < n; ++col) R[(size_t)lp * n + col] *= std::conj(e);
                    cd acc = 0;
                    for (int col = 0; col < n; ++col) acc += M[(size_t)lp * n + col] * R[(size_t)lp * n + col];
                    grad[aidx[seq[kk]]] += (acc * I * e).real();
                    for (int col = 0; col < n; ++col) M[(size_t)lp * n + col] *= e;
                }
            }
        }
    }
}

int grad_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, const double* d_grad_p, double* d_out_p,
             std::vector<double>& grad, cudaStream_t s) {
    if (!c->exact_ok) return fail(EF_EUNSUPPORTED, c->exact_why);
    for (int b = 0; b < c->nblocks; ++b) {
        const HostBlock& B = c->blk[b];
        if (B.eta > 8 || B.n > 64 || ef::grad_minors_smem(B.n, B.eta, B.L) > 227 * 1024)
            return fail(EF_EUNSUPPORTED, "ef_prob_grad: supports mode blocks of at most 64 modes and 8 particles "
                                         "(and layers x modes x particles within shared memory)");
    }
    int rc = begin_call(c, s, 3);
    if (rc) return rc;
    int64_t na = 0;
    for (const ef_gate& g : c->gates) na += g.kind == EF_GIVENS ? 2 : 1;
    grad.assign(na, 0.0);
    c->stats.logical_branch_dets = nb * (int64_t)std::ldexp(1.0, (int)c->cps.size());
    if (nb == 0) return EF_OK;
    ef::LaunchStats st;
    const int ksh = c->nblocks == 2 ? (int)c->shared_gates.size() : 0;
    size_t need = 0;
    for (int b = 0; b < c->nblocks; ++b) {
        const HostBlock& B = c->blk[b];
        const size_t ny = (size_t)1 << B.r;
        need += ny * (size_t)nb * (2 * sizeof(double2)) + (size_t)nb * ((size_t)1 << B.r_loc) * 16 +
                ny * ((size_t)B.L * B.n * B.n + (size_t)B.n * B.eta) * 16;
    }
    need += (size_t)nb * ((size_t)1 << ksh) * 16;
    if (need > ((size_t)24 << 30))
        return fail(EF_EUNSUPPORTED, "ef_prob_grad: the call needs " + std::to_string(need >> 20) +
                                         " MiB of device workspace; split the bitstrings into smaller calls");
    ef::GradDev g{};
    ef::ExactCombineDev& cm = g.cm;
    cm.nblocks = c->nblocks;
    cm.k_sh = ksh;
    cm.inactive0 = c->inactive[0];
    cm.inactive1 = c->inactive[1];
    cm.WS = c->dWS.as<double2>();
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const size_t ny = (size_t)1 << B.r;
        const size_t ne = (size_t)B.n * B.eta;
        EF_CK(B.dM64.ensure(ny * ne * sizeof(double2)));
        EF_CK(B.dD64.ensure(ny * (size_t)nb * sizeof(double2)));
        EF_CK(B.dCot.ensure(ny * (size_t)nb * sizeof(double2)));
        EF_CK(B.dEbar.ensure((size_t)nb * ((size_t)1 << B.r_loc) * sizeof(double2)));
        EF_CK(B.dTbar.ensure(ny * std::max<size_t>(1, (size_t)B.L * B.n * B.n) * sizeof(double2)));
        EF_CK(B.dSbar.ensure(ny * ne * sizeof(double2)));
        EF_CK(B.dSumT.ensure(std::max<size_t>(1, (size_t)B.L * B.n * B.n) * sizeof(double2)));
        EF_CK(B.dSumS.ensure(ne * sizeof(double2)));
        EF_CK(B.dSumE.ensure(((size_t)1 << B.r_loc) * sizeof(double2)));
        ef::ExactBlockDev& d = g.blk[b];
        exact_block_geometry(c, b, nb, d);
        d.S0C = B.dS0C.as<double2>();
        d.T = B.dT.as<double2>();
        d.F = B.dF.as<uint32_t>();
        d.M64 = B.dM64.as<double2>();
        d.M32 = nullptr;
        d.ML32 = nullptr;
        d.D32 = nullptr;
        d.E32 = nullptr;
        d.D64 = B.dD64.as<double2>();
        cm.mask[b][0] = B.mask[0];
        cm.mask[b][1] = B.mask[1];
        cm.eta[b] = B.eta;
        cm.r[b] = B.r;
        cm.r_loc[b] = B.r_loc;
        cm.D64[b] = d.D64;
        cm.src = 1;
        cm.Omega[b] = B.dOmega.as<double2>();
        cm.s[b] = B.dSh.as<uint32_t>();
        cm.perm[b] = B.dPerm.as<uint32_t>();
        cm.goff[b] = B.dGoff.as<uint32_t>();
        g.cot[b] = B.dCot.as<double2>();
        g.ebar[b] = B.dEbar.as<double2>();
        g.tbar[b] = B.dTbar.as<double2>();
        g.sbar[b] = B.dSbar.as<double2>();
    }
    EF_CK(c->dPbar.ensure((size_t)nb * ((size_t)1 << ksh) * sizeof(double2)));
    EF_CK(c->dSumP.ensure(((size_t)1 << ksh) * sizeof(double2)));
    g.pbar = c->dPbar.as<double2>();
    if (c->nblocks > 0) EF_CK(ef::launch_build_branches(g.blk[0], g.blk[1], c->nblocks, false, s, st));
    for (int b = 0; b < c->nblocks; ++b) EF_CK(ef::launch_exact_lu_f64(g.blk[b], d_bits, nb, nullptr, nullptr, nb, s, st));
    if (c->timed) EF_CK(cudaEventRecord(c->ev0, s));
    EF_CK(ef::launch_grad(g, d_bits, nb, d_grad_p, d_out_p, s, st));
    if (c->timed) EF_CK(cudaEventRecord(c->ev1, s));
    c->stats.dominant_kernel_launches = 1 + c->nblocks;
    std::vector<std::vector<cd>> tbar(c->nblocks), sbar(c->nblocks), ebar(c->nblocks);
    std::vector<cd> pbar;
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const int64_t ny = (int64_t)1 << B.r;
        const int64_t wT = (int64_t)B.L * B.n * B.n, wS = (int64_t)B.n * B.eta, wE = (int64_t)1 << B.r_loc;
        EF_CK(ef::launch_sum_rows(B.dTbar.as<double2>(), ny, wT, wT, B.dSumT.as<double2>(), s, st));
        EF_CK(ef::launch_sum_rows(B.dSbar.as<double2>(), ny, wS, wS, B.dSumS.as<double2>(), s, st));
        EF_CK(ef::launch_sum_rows(B.dEbar.as<double2>(), nb, wE, wE, B.dSumE.as<double2>(), s, st));
        tbar[b].resize(wT);
        sbar[b].resize(wS);
        ebar[b].resize(wE);
        if (wT) EF_CK(cudaMemcpyAsync(tbar[b].data(), B.dSumT.p, wT * sizeof(double2), cudaMemcpyDeviceToHost, s));
        EF_CK(cudaMemcpyAsync(sbar[b].data(), B.dSumS.p, wS * sizeof(double2), cudaMemcpyDeviceToHost, s));
        EF_CK(cudaMemcpyAsync(ebar[b].data(), B.dSumE.p, wE * sizeof(double2), cudaMemcpyDeviceToHost, s));
    }
    if (c->nblocks == 2) {
        const int64_t wP = (int64_t)1 << ksh;
        EF_CK(ef::launch_sum_rows(c->dPbar.as<double2>(), nb, wP, wP, c->dSumP.as<double2>(), s, st));
        pbar.resize(wP);
        EF_CK(cudaMemcpyAsync(pbar.data(), c->dSumP.p, wP * sizeof(double2), cudaMemcpyDeviceToHost, s));
    }
    EF_CK(cudaStreamSynchronize(s));
    c->stats.kernel_launches = st.launches;
    c->stats.executed_minor_lus = 2 * st.executed_lus;
    grad_finish(c, tbar, sbar, ebar, pbar, grad);
    return EF_OK;
}

// Buffers and launch parameters of a Raw Estimate call (no stream work).
// Items are (bitstring, chunk of trajectories): one chunk per bitstring when
// the bitstrings alone fill the GPU, more otherwise; CTAs stride over them.
// The K form is used when every block has at most 64 flippable pairs and the
// CTA's shared memory fits; otherwise every flipped minor takes the rank-one
// form.
ef::ApproxDev approx_dev_for(const ef_circuit* c, const ef::ApproxDev& base, bool fp64) {
    ef::ApproxDev a = base;
    for (int b = 0; b < c->nblocks; ++b) {
        const HostBlock& B = c->blk[b];
        a.blk[b].P = fp64 ? B.dP64.p : B.dP32.p;
        a.blk[b].RC = fp64 ? B.dRC64.p : B.dRC32.p;
    }
    a.kform = c->kform_ok ? 1 : 0;
    const int eta_t = ef::approx_eta_template(a);
    if (a.kform && ef::approx_smem_bytes(a, eta_t, fp64) > (size_t)200 * 1024) a.kform = 0;
    a.err_coef = fp64 ? 0.0 : base.err_coef;
    a.err_lin = fp64 ? 0.0 : base.err_lin;
    return a;
}

int approx_setup(ef_circuit* c, int64_t nb, int64_t t, uint64_t seed, uint64_t base, ef::ApproxDev& a) {
    if (!c->approx_ok) return fail(EF_EUNSUPPORTED, c->approx_why);
    const bool fp64 = c->opt.precision == EF_PREC_FP64;
    if (fp64)
        for (int b = 0; b < c->nblocks; ++b)
            if (c->blk[b].eta > ef::kMaxApproxEta64)
                return fail(EF_EUNSUPPORTED, "Raw Estimate with FP64 minors: at most 13 particles per mode block");
    if (t <= 0 || t > (int64_t)4294967296ll) return fail(EF_EINVAL, "n_traj must be in 1..2^32");
    if (nb > 2147483647ll) return fail(EF_EUNSUPPORTED, "Raw Estimate: more than 2^31-1 bitstrings per call");
    a = ef::ApproxDev{};
    a.nblocks = c->nblocks;
    a.k = (int)c->cps.size();
    a.T = c->daT.as<uint32_t>();
    a.qratio = c->daq.as<double>();
    a.qratio32 = c->daq32.as<float>();
    a.glayer = c->dalayer.as<uint8_t>();
    a.gmodes = c->damodes.as<uint64_t>();
    a.gpair = c->dagpair.as<uint64_t>();
    a.R0 = c->R0;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.index_base = base;
    a.inactive0 = c->inactive[0];
    a.inactive1 = c->inactive[1];
    a.t = t;
    a.nb = nb;
    // enough (bitstring, chunk) items for about four waves of three CTAs per SM
    const int64_t sms = ef::sm_count();
    const int64_t target = sms * 3 * 4;
    int64_t chunks = std::max<int64_t>(1, (target + std::max<int64_t>(nb, 1) - 1) / std::max<int64_t>(nb, 1));
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, t / 256));
    int64_t per = (t + chunks - 1) / chunks;
    per = (per + 127) / 128 * 128;
    a.traj_per_cta = (int)std::min<int64_t>(per, (int64_t)1 << 30);
    a.n_chunks = (int)((t + a.traj_per_cta - 1) / a.traj_per_cta);
    // one CTA per item (the hardware balances them); the listed FP64 redo strides
    a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(nb, 1) * a.n_chunks, 2147483647ll));
    a.kappa_max = 1e3;
    // K u, the per-trajectory bounds being in units of u = 2^-24. Calibrated
    // against FP64 on the same trajectories (eight circuits, 12,226 results: the
    // 52-qubit LUCJ workload, the parity-test circuits, Raw Estimate circuits of
    // the 64-circuit batch): the largest observed error / estimate was 0.22 at
    // K = 0.5 with n_max taken from the most probable flipped trajectory. With
    // the pair-based n_max below and the rank-one form's bounds summed
    // linearly, the largest ratio over the 26 Raw Estimate circuits of that
    // batch (69,727 results) is 0.45.
    a.err_coef = 0.5 * std::ldexp(1.0, -24);
    a.err_lin = std::ldexp(1.0, -24);
    // How many trajectories share one rounded quantity: a small determinant
    // (its flipped pairs), an entry of K (every trajectory flipping its pair),
    // a whole trajectory. Each count is at most that of trajectories flipping
    // one given pair, so the largest probability that a pair is flipped
    // bounds them all: pair a of block B flips when an odd number of the gates
    // that flip it do, P = (1 - prod_j (1 - 2 pT1_j)) / 2. Without the K form
    // (no pair tables) the most probable flipped trajectory is used instead:
    // x* with x_j = [pT1_j > 1/2] if it flips a gate, else the single flip
    // with the largest pT1/pT0 added to x = 0.
    {
        double logp = 0.0, best_ratio = 0.0;
        bool any = false;
        for (const CP& cp : c->cps) {
            if (cp.pT1 > 0.5) any = true;
            logp += std::log(std::max(cp.pT1, cp.pT0));
            if (cp.pT1 <= 0.5 && cp.pT0 > 0.0) best_ratio = std::max(best_ratio, cp.pT1 / cp.pT0);
        }
        double q = any ? std::exp(logp) : std::exp(logp) * best_ratio;
        if (c->kform_ok) {
            const int k = (int)c->cps.size();
            for (int b = 0; b < c->nblocks; ++b)
                for (int pp = 0; pp < 64; ++pp) {
                    double even = 1.0;  // prod_j (1 - 2 pT1_j) over the gates flipping pair pp
                    bool touched = false;
                    for (int jj = 0; jj < k; ++jj)
                        if ((c->agpair[(size_t)b * k + jj] >> pp) & 1ull) {
                            even *= 1.0 - 2.0 * c->cps[jj].pT1;
                            touched = true;
                        }
                    if (touched) q = std::max(q, 0.5 * (1.0 - even));
                }
        }
        const double mean = (double)t * q;
        a.nmax = std::max(1.0, mean + 3.0 * std::sqrt(mean) + 1.0);
    }
    a.tol = c->opt.tol;
    a.p_floor = c->p_floor;
    EF_CK(c->daPart.ensure((size_t)std::max<int64_t>(nb, 1) * a.n_chunks * ef::kApproxPartStride * sizeof(double)));
    EF_CK(c->dCounters.ensure(8 * sizeof(unsigned long long)));
    EF_CK(c->daList.ensure(((size_t)std::max<int64_t>(nb, 1) + 4) * sizeof(int)));
    a.part = c->daPart.as<double>();
    a.counters = c->dCounters.as<unsigned long long>();
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        a.blk[b].n = B.n;
        a.blk[b].eta = B.eta;
        a.blk[b].L = B.L;
        a.blk[b].mask0 = B.mask[0];
        a.blk[b].mask1 = B.mask[1];
        a.blk[b].P64 = B.dP64.as<double2>();
        a.blk[b].RC64 = B.dRC64.as<double2>();
        a.blk[b].cols = B.dCols.as<int>();
        a.blk[b].f = (int)B.pair_lm.size();
        a.blk[b].pair_lm = B.dPairLM.as<int>();
    }
    a = approx_dev_for(c, a, fp64);
    return EF_OK;
}

// The Raw Estimate launches: trajectories, finalisation and, under
// EF_PREC_AUTO, the FP64 redo of the bitstrings whose estimated relative
// error exceeds tol (same seed and global indices, so the same trajectories).
int approx_enqueue(ef_circuit* c, const ef::ApproxDev& a, const uint64_t* d_bits, double* d_out, double* d_se,
                   double* d_err, cudaStream_t s, ef::LaunchStats& st) {
    const bool fp64 = c->opt.precision == EF_PREC_FP64;
    const bool autofix = c->opt.precision == EF_PREC_AUTO && ef::approx_eta_template(a) <= ef::kMaxApproxEta64;
    int* list = c->daList.as<int>();
    int* list_count = list + std::max<int64_t>(a.nb, 1);
    EF_CK(cudaMemsetAsync(a.counters, 0, 8 * sizeof(unsigned long long), s));
    EF_CK(cudaMemsetAsync(list_count, 0, sizeof(int), s));
    if (c->timed) EF_CK(cudaEventRecord(c->ev0, s));
    EF_CK(ef::launch_approx(a, d_bits, fp64, s, st));
    if (c->timed) EF_CK(cudaEventRecord(c->ev1, s));
    EF_CK(ef::launch_approx_finalize(a, d_out, d_se, d_err, autofix ? list : nullptr, list_count, false, s, st));
    if (autofix) {
        ef::ApproxDev r = approx_dev_for(c, a, true);
        r.list = list;
        r.list_count = list_count;
        r.counters = a.counters + 4;  // the redo's own flips, LUs and rank-one minors
        r.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)a.grid, (int64_t)ef::sm_count() * 24));
        EF_CK(ef::launch_approx(r, d_bits, true, s, st));
        EF_CK(ef::launch_approx_finalize(r, d_out, d_se, d_err, nullptr, nullptr, true, s, st));
    }
    return EF_OK;
}

int approx_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, int64_t t, uint64_t seed, uint64_t base,
               double* d_out, double* d_se, double* d_err, cudaStream_t s) {
    if (!c->approx_ok) return fail(EF_EUNSUPPORTED, c->approx_why);
    if (t <= 0 || t > (int64_t)4294967296ll) return fail(EF_EINVAL, "n_traj must be in 1..2^32");
    int rc = begin_call(c, s, 2);
    if (rc) return rc;
    c->stats.logical_branch_dets = nb * t;
    if (nb == 0) return EF_OK;
    ef::ApproxDev a;
    rc = approx_setup(c, nb, t, seed, base, a);
    if (rc) return rc;
    ef::LaunchStats st;
    rc = approx_enqueue(c, a, d_bits, d_out, d_se, d_err, s, st);
    if (rc) return rc;
    c->stats.dominant_kernel_launches = 1;
    c->stats.kernel_launches = st.launches;
    return EF_OK;
}

// ------------------------------------------------------------------ Estimate (Section III-A)

// Eq. 6: trajectories sufficient for |p_hat - p| <= eps with failure
// probability at most delta when p <= p_max (the printed "= 1 - delta" read as
// "<= delta"), before rounding up.
double trajectory_bound(double eps, double delta, double pmax, double xi) {
    const double num = std::sqrt(xi) + std::sqrt(pmax);
    const double den = std::sqrt(pmax + eps) - std::sqrt(pmax);
    const double e = 2.718281828459045;
    return std::ceil(2.0 * (num * num) / (den * den) * std::log(2.0 * (e * e) / delta));
}

// Trajectory counts are rounded up to m * 2^e with 4 <= m <= 8 (at most 25 %
// more), so that the bitstrings of a round fall into a few shared launches.
int64_t trajectory_grid(int64_t t) {
    if (t <= 8) return std::max<int64_t>(t, 1);
    int len = 0;
    while (len < 63 && (t >> len) != 0) ++len;
    const int e = len - 3;
    const int64_t m = (t + ((int64_t)1 << e) - 1) >> e;
    return m << e;
}

// SplitMix64 (Steele, Lea and Flood 2014): the seed of round r is
// splitmix64(seed + (r + 1) * 0x9E3779B97F4A7C15), so rounds draw independent trajectories.
uint64_t splitmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bool bitstring_in_sector(const ef_circuit* c, uint64_t w0, uint64_t w1) {
    if ((w0 & c->inactive[0]) || (w1 & c->inactive[1])) return false;
    for (int b = 0; b < c->nblocks; ++b)
        if (__builtin_popcountll(w0 & c->blk[b].mask[0]) + __builtin_popcountll(w1 & c->blk[b].mask[1]) !=
            c->blk[b].eta)
            return false;
    return true;
}

// The Estimate algorithm as rounds of Raw Estimate. Round r = 0 .. R-1 runs
// every bitstring with eps_r = max(eps, eps_0 / 2^r) (eps_0 = max(eps, 1/4),
// R the first round with eps_r = eps), delta_r = delta / R and the Eq. 6 count
// for its own bound p_max (1 at the start), then tightens p_max to
// min(p_max, p_hat + eps_r); the last round's p_hat is the estimate. Every
// round holds its guarantee with probability >= 1 - delta_r, so all of them do
// (and the final |p_hat - p| <= eps) with probability >= 1 - delta.
int estimate_host(ef_circuit* c, const uint64_t* bits, int64_t nb, double eps, double delta, uint64_t seed,
                  uint64_t index_base, double* out, double* se_out, int64_t* traj_out) {
    const double eps0 = std::max(eps, 0.25);
    int R = 1;
    while (R < 64 && std::max(eps, std::ldexp(eps0, -(R - 1))) > eps) ++R;
    const double delta_r = delta / R;
    std::vector<double> pmax(nb, 1.0), ph(nb, 0.0), se(nb, 0.0);
    std::vector<int64_t> traj(nb, 0);
    std::vector<char> valid(nb);
    for (int64_t i = 0; i < nb; ++i) valid[i] = bitstring_in_sector(c, bits[2 * i], bits[2 * i + 1]);
    if (!c->own_stream) EF_CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    const cudaStream_t s = c->own_stream;
    DBuf dbits, didx, dout;
    EF_CK(dbits.ensure((size_t)std::max<int64_t>(nb, 1) * 2 * sizeof(uint64_t)));
    EF_CK(didx.ensure((size_t)std::max<int64_t>(nb, 1) * sizeof(uint64_t)));
    EF_CK(dout.ensure((size_t)std::max<int64_t>(nb, 1) * 2 * sizeof(double)));
    ef_stats total{};
    std::vector<uint64_t> gb, gi;
    std::vector<double> gp, gs;
    for (int r = 0; r < R; ++r) {
        const double eps_r = std::max(eps, std::ldexp(eps0, -r));
        const uint64_t seed_r = splitmix64(seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull);
        std::map<int64_t, std::vector<int64_t>> groups;
        for (int64_t i = 0; i < nb; ++i) {
            if (!valid[i]) continue;
            const double tb = trajectory_bound(eps_r, delta_r, pmax[i], c->xi);
            if (!(tb <= 4294967296.0))
                return fail(EF_EUNSUPPORTED, "ef_prob_estimate: round " + std::to_string(r) + " needs more than 2^32 "
                                             "trajectories for bitstring " + std::to_string(i));
            groups[trajectory_grid((int64_t)tb)].push_back(i);
        }
        for (auto& kv : groups) {
            const int64_t t = std::min<int64_t>(kv.first, (int64_t)4294967296ll);
            const std::vector<int64_t>& ids = kv.second;
            const int64_t ng = (int64_t)ids.size();
            gb.resize(2 * ng);
            gi.resize(ng);
            for (int64_t j = 0; j < ng; ++j) {
                gb[2 * j] = bits[2 * ids[j]];
                gb[2 * j + 1] = bits[2 * ids[j] + 1];
                gi[j] = index_base + (uint64_t)ids[j];
            }
            EF_CK(cudaMemcpyAsync(dbits.p, gb.data(), gb.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
            EF_CK(cudaMemcpyAsync(didx.p, gi.data(), gi.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
            int rc = begin_call(c, s, 2);
            if (rc) return rc;
            ef::ApproxDev a;
            rc = approx_setup(c, ng, t, seed_r, 0, a);
            if (rc) return rc;
            a.gidx = didx.as<uint64_t>();
            ef::LaunchStats st;
            double* d_p = dout.as<double>();
            rc = approx_enqueue(c, a, dbits.as<uint64_t>(), d_p, d_p + ng, nullptr, s, st);
            if (rc) return rc;
            gp.resize(ng);
            gs.resize(ng);
            EF_CK(cudaMemcpyAsync(gp.data(), d_p, ng * sizeof(double), cudaMemcpyDeviceToHost, s));
            EF_CK(cudaMemcpyAsync(gs.data(), d_p + ng, ng * sizeof(double), cudaMemcpyDeviceToHost, s));
            unsigned long long h[8] = {};
            EF_CK(cudaMemcpyAsync(h, a.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
            EF_CK(cudaStreamSynchronize(s));
            for (int64_t j = 0; j < ng; ++j) {
                const int64_t i = ids[j];
                ph[i] = gp[j];
                se[i] = gs[j];
                pmax[i] = std::min(pmax[i], gp[j] + eps_r);
                traj[i] += t;
            }
            total.logical_branch_dets += ng * t;
            total.sampled_flips += (int64_t)h[0];
            total.executed_minor_lus += (int64_t)(h[1] + h[5]);
            total.fp64_recomputed += (int64_t)h[3];
            total.kernel_launches += st.launches;
        }
    }
    for (int64_t i = 0; i < nb; ++i) {
        out[i] = ph[i];
        if (se_out) se_out[i] = se[i];
        if (traj_out) traj_out[i] = traj[i];
    }
    cudaStreamSynchronize(s);
    dbits.release();
    didx.release();
    dout.release();
    c->stats = total;
    c->last_mode = 0;
    return EF_OK;
}

// Host-pointer form of a *_dev call: bitstrings in, up to three per-bitstring
// outputs back (out2, out3 nullable), on the circuit's own stream.
int check_bits_host(const ef_circuit* c, const uint64_t* bits, int64_t nb) {
    uint64_t hi[2] = {0, 0};
    if (c->n < 64) hi[0] = ~0ull << c->n, hi[1] = ~0ull;
    else if (c->n < 128) hi[1] = ~0ull << (c->n - 64);
    for (int64_t i = 0; i < nb; ++i)
        if ((bits[2 * i] & hi[0]) || (bits[2 * i + 1] & hi[1]))
            return fail(EF_EINVAL, "bitstring " + std::to_string(i) + " has a bit at or above n_modes");
    return EF_OK;
}

template <typename F>
int host_call(ef_circuit* c, const uint64_t* bits, int64_t nb, double* out, double* out2, double* out3,
              F&& dev_call) {
    if (!c->own_stream) EF_CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    cudaStream_t s = c->own_stream;
    if (nb > 0) {
        EF_CK(c->dBits.ensure((size_t)nb * 2 * sizeof(uint64_t)));
        EF_CK(c->dOut.ensure((size_t)nb * 3 * sizeof(double)));
        EF_CK(cudaMemcpyAsync(c->dBits.p, bits, (size_t)nb * 2 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    }
    double* d0 = c->dOut.as<double>();
    double* d2 = out2 ? d0 + nb : nullptr;
    double* d3 = out3 ? d0 + 2 * nb : nullptr;
    int rc = dev_call(c->dBits.as<uint64_t>(), d0, d2, d3, s);
    if (rc) return rc;
    // the host-side argument check runs while the GPU works (the kernels only
    // read the bits through the blocks' mode masks, so a bit at or above n
    // cannot make them access memory out of range); on failure nothing is
    // copied back
    rc = check_bits_host(c, bits, nb);
    if (rc) {
        cudaStreamSynchronize(s);
        return rc;
    }
    if (nb > 0) {
        EF_CK(cudaMemcpyAsync(out, d0, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (out2) EF_CK(cudaMemcpyAsync(out2, d2, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (out3) EF_CK(cudaMemcpyAsync(out3, d3, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    EF_CK(cudaStreamSynchronize(s));
    return EF_OK;
}


}  // namespace

// =================================================================== C ABI

extern "C" {

int ef_version(void) { return 100; }

const char* ef_last_error(void) { return g_err.c_str(); }

int ef_circuit_create(int32_t n_modes, const uint64_t occupation[2], const ef_gate* gates, int64_t n_gates,
                      const ef_options* opt, ef_circuit** out) {
    if (!out) return fail(EF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!occupation) return fail(EF_EINVAL, "occupation is NULL");
    if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(EF_EINVAL, "bad gate list");
    if (n_modes < 1 || n_modes > ef::kMaxModes) return fail(EF_EINVAL, "n_modes must be in 1..128");
    uint64_t hi[2] = {0, 0};
    if (n_modes < 64) hi[0] = ~0ull << n_modes, hi[1] = ~0ull;
    else if (n_modes < 128) hi[1] = ~0ull << (n_modes - 64);
    if ((occupation[0] & hi[0]) || (occupation[1] & hi[1])) return fail(EF_EINVAL, "occupation has a bit at or above n_modes");
    int rc = validate_gates(n_modes, gates, n_gates);
    if (rc) return rc;
    ef_circuit* c = new (std::nothrow) ef_circuit();
    if (!c) return fail(EF_ENOMEM, "host allocation failed");
    static std::atomic<uint64_t> next_uid{1};
    c->uid = next_uid++;
    c->n = n_modes;
    c->occ[0] = occupation[0];
    c->occ[1] = occupation[1];
    c->gates.assign(gates, gates + n_gates);
    c->opt.precision = EF_PREC_AUTO;
    c->opt.flags = 0;
    c->opt.tol = 1e-5;
    if (opt) {
        c->opt = *opt;
        if (c->opt.precision < 0 || c->opt.precision > 2) {
            delete c;
            return fail(EF_EINVAL, "bad precision");
        }
        if (!(c->opt.tol > 0)) c->opt.tol = 1e-5;
    }
    // the device is only needed by the probability calls; creation and the host
    // preprocessing work without one
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        c->device = -1;
        cudaGetLastError();
    }
    rc = prepare(c);
    if (rc) {
        delete c;
        return rc;
    }
    *out = c;
    return EF_OK;
}

int ef_circuit_destroy(ef_circuit* c) {
    if (!c) return EF_OK;
    if (c->has_last_stream) cudaStreamSynchronize(c->last_stream);
    delete c;
    return EF_OK;
}

int ef_circuit_num_angles(const ef_circuit* c, int64_t* n) {
    if (!c || !n) return fail(EF_EINVAL, "NULL argument");
    int64_t k = 0;
    for (const ef_gate& g : c->gates) k += g.kind == EF_GIVENS ? 2 : 1;
    *n = k;
    return EF_OK;
}

int ef_circuit_get_angles(const ef_circuit* c, double* angles, int64_t n) {
    int64_t k;
    int rc = ef_circuit_num_angles(c, &k);
    if (rc) return rc;
    if (n != k || (k > 0 && !angles)) return fail(EF_EINVAL, "angle count mismatch");
    int64_t i = 0;
    for (const ef_gate& g : c->gates) {
        if (g.kind == EF_GIVENS) {
            angles[i++] = g.theta;
            angles[i++] = g.phi;
        } else if (g.kind == EF_PHASE) {
            angles[i++] = g.phi;
        } else {
            angles[i++] = g.theta;
        }
    }
    return EF_OK;
}

int ef_circuit_set_angles(ef_circuit* c, const double* angles, int64_t n) {
    int64_t k;
    int rc = ef_circuit_num_angles(c, &k);
    if (rc) return rc;
    if (n != k || (k > 0 && !angles)) return fail(EF_EINVAL, "angle count mismatch");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(angles[i])) return fail(EF_EINVAL, "non-finite angle");
    if (c->has_last_stream) EF_CK(cudaStreamSynchronize(c->last_stream));
    int64_t i = 0;
    for (ef_gate& g : c->gates) {
        if (g.kind == EF_GIVENS) {
            g.theta = angles[i++];
            g.phi = angles[i++];
        } else if (g.kind == EF_PHASE) {
            g.phi = angles[i++];
        } else {
            g.theta = angles[i++];
        }
    }
    return prepare(c);
}

int ef_circuit_extent(const ef_circuit* c, double* xi) {
    if (!c || !xi) return fail(EF_EINVAL, "NULL argument");
    *xi = c->xi;
    return EF_OK;
}

int ef_circuit_set_precision(ef_circuit* c, int32_t precision, double tol) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (precision < 0 || precision > 2) return fail(EF_EINVAL, "bad precision");
    if (c->has_last_stream) EF_CK(cudaStreamSynchronize(c->last_stream));
    c->opt.precision = precision;
    if (tol > 0) c->opt.tol = tol;
    return EF_OK;
}

int ef_prob_exact_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, double* d_out, double* d_err_out,
                      void* stream) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!d_bits || !d_out))) return fail(EF_EINVAL, "bad bitstring/output arguments");
    if (nb > 2147483647ll) return fail(EF_EUNSUPPORTED, "more than 2^31-1 bitstrings per call");
    return exact_dev(c, d_bits, nb, d_out, d_err_out, (cudaStream_t)stream);
}

int ef_prob_exact(ef_circuit* c, const uint64_t* bits, int64_t nb, double* out, double* err_out) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!bits || !out))) return fail(EF_EINVAL, "bad bitstring/output arguments");
    return host_call(c, bits, nb, out, err_out, nullptr,
                     [&](const uint64_t* db, double* dout, double* derr, double*, cudaStream_t s) {
                         return ef_prob_exact_dev(c, db, nb, dout, derr, s);
                     });
}

int ef_prob_approx_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, int64_t n_traj, uint64_t seed,
                       uint64_t index_base, double* d_out, double* d_stderr_out, double* d_err_out, void* stream) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!d_bits || !d_out))) return fail(EF_EINVAL, "bad bitstring/output arguments");
    return approx_dev(c, d_bits, nb, n_traj, seed, index_base, d_out, d_stderr_out, d_err_out, (cudaStream_t)stream);
}

int ef_prob_approx(ef_circuit* c, const uint64_t* bits, int64_t nb, int64_t n_traj, uint64_t seed,
                   uint64_t index_base, double* out, double* stderr_out, double* err_out) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!bits || !out))) return fail(EF_EINVAL, "bad bitstring/output arguments");
    return host_call(c, bits, nb, out, stderr_out, err_out,
                     [&](const uint64_t* db, double* dout, double* dse, double* derr, cudaStream_t s) {
                         return ef_prob_approx_dev(c, db, nb, n_traj, seed, index_base, dout, dse, derr, s);
                     });
}

int ef_prob_estimate(ef_circuit* c, const uint64_t* bits, int64_t nb, double eps, double delta, uint64_t seed,
                     uint64_t index_base, double* out, double* stderr_out, int64_t* traj_out) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!bits || !out))) return fail(EF_EINVAL, "bad bitstring/output arguments");
    if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) return fail(EF_EINVAL, "need eps > 0 and 0 < delta < 1");
    if (!c->approx_ok) return fail(EF_EUNSUPPORTED, c->approx_why);
    int rc = check_bits_host(c, bits, nb);
    if (rc) return rc;
    if (nb == 0) return EF_OK;
    return estimate_host(c, bits, nb, eps, delta, seed, index_base, out, stderr_out, traj_out);
}

int ef_prob_grad_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, const double* d_grad_p, double* d_out_p,
                     double* d_grad_angles, void* stream) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!d_bits || !d_grad_p)) || !d_grad_angles)
        return fail(EF_EINVAL, "bad bitstring/gradient arguments");
    if (nb > 2147483647ll) return fail(EF_EUNSUPPORTED, "more than 2^31-1 bitstrings per call");
    std::vector<double> grad;
    const cudaStream_t s = (cudaStream_t)stream;
    int rc = grad_dev(c, d_bits, nb, d_grad_p, d_out_p, grad, s);
    if (rc) return rc;
    if (!grad.empty()) {
        EF_CK(cudaMemcpyAsync(d_grad_angles, grad.data(), grad.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        EF_CK(cudaStreamSynchronize(s));
    }
    return EF_OK;
}

int ef_prob_grad(ef_circuit* c, const uint64_t* bits, int64_t nb, const double* grad_p, double* out_p,
                 double* grad_angles) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!bits || !grad_p)) || !grad_angles) return fail(EF_EINVAL, "bad arguments");
    int rc = check_bits_host(c, bits, nb);
    if (rc) return rc;
    if (!c->own_stream) EF_CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    const cudaStream_t s = c->own_stream;
    if (nb > 0) {
        EF_CK(c->dBits.ensure((size_t)nb * 2 * sizeof(uint64_t)));
        EF_CK(c->dGradP.ensure((size_t)nb * sizeof(double)));
        EF_CK(c->dOut.ensure((size_t)nb * sizeof(double)));
        EF_CK(cudaMemcpyAsync(c->dBits.p, bits, (size_t)nb * 2 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        EF_CK(cudaMemcpyAsync(c->dGradP.p, grad_p, (size_t)nb * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    std::vector<double> grad;
    rc = grad_dev(c, c->dBits.as<uint64_t>(), nb, c->dGradP.as<double>(), nb > 0 ? c->dOut.as<double>() : nullptr,
                  grad, s);
    if (rc) return rc;
    if (out_p && nb > 0) {
        EF_CK(cudaMemcpyAsync(out_p, c->dOut.p, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        EF_CK(cudaStreamSynchronize(s));
    }
    std::copy(grad.begin(), grad.end(), grad_angles);
    return EF_OK;
}

int ef_circuit_get_stats(ef_circuit* c, ef_stats* st) {
    if (!c || !st) return fail(EF_EINVAL, "NULL argument");
    if (c->has_last_stream) EF_CK(cudaStreamSynchronize(c->last_stream));
    if (c->timed && c->ev0 && c->stats.dominant_kernel_launches > 0) {
        float ms = 0.f;
        EF_CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        c->stats.dominant_kernel_ms = ms;
    }
    if (c->last_mode == 1 && c->last_fp64_list_pending && c->last_recomp) {
        unsigned long long cnt[2] = {0, 0};
        EF_CK(cudaMemcpy(cnt, c->last_recomp, sizeof(cnt), cudaMemcpyDeviceToHost));
        c->stats.fp64_recomputed = (int64_t)cnt[0];
        c->stats.executed_minor_lus += (int64_t)cnt[1];
        c->last_fp64_list_pending = 0;
    }
    if (c->last_mode == 2 && c->dCounters.p) {
        unsigned long long h[4] = {0, 0, 0, 0};
        EF_CK(cudaMemcpy(h, c->dCounters.p, sizeof(h), cudaMemcpyDeviceToHost));
        unsigned long long r[2] = {0, 0};
        EF_CK(cudaMemcpy(r, c->dCounters.as<unsigned long long>() + 4, sizeof(r), cudaMemcpyDeviceToHost));
        c->stats.sampled_flips = (int64_t)h[0];
        c->stats.executed_minor_lus = (int64_t)h[1] + (int64_t)r[1];
        c->stats.fp64_recomputed = (int64_t)h[3];
    }
    *st = c->stats;
    return EF_OK;
}

}  // extern "C"

// =================================================================== allocation-free Exact entry point
//
// ef_prob_exact_noalloc_dev runs the same kernels as ef_prob_exact_dev but
// takes every device buffer it needs (circuit tables, branch matrices,
// partial sums, the recompute list) from one fixed array that the library
// declares at file scope. It is for callers that must not have a library
// allocate device memory during their run (see extraferm.h).

#include <mutex>

namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // 64 MiB per GPU, held until the process exits
constexpr int kNoAllocMaxDevices = 64;

// File-scope scratch. In host code this name is only a stand-in for the
// device symbol; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};
// whose tables the scratch of each device holds: (circuit uid, table generation)
uint64_t g_noalloc_owner[kNoAllocMaxDevices][2] = {};

// Device address of the scratch on the current device (set up once per device).
int noalloc_base(unsigned char** out) {
    int dev = -1;
    EF_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(EF_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(EF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return EF_OK;
}

__global__ void k_gather_columns(const double2* __restrict__ S0, const int* __restrict__ cols, int n, int eta,
                                 double2* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * eta; e += gridDim.x * blockDim.x) {
        const int i = e / eta, c = e - i * eta;
        out[e] = S0[(size_t)i * n + cols[c]];
    }
}

// Carves 256-byte aligned regions out of the scratch; only sizes on the first pass.
struct Carver {
    unsigned char* base;
    size_t off = 0;
    template <typename T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

struct NoAllocTables {
    double2* S0[ef::kMaxBlocks];
    int* cols[ef::kMaxBlocks];
};

// The circuit's tables come first (their offsets depend on the circuit only,
// so a later call on the same circuit finds them in place), then the buffers
// sized by the call.
size_t noalloc_layout(ef_circuit* c, int64_t nb, bool want32, unsigned char* base, ExactBuffers& eb,
                      NoAllocTables& tb) {
    Carver cv{base};
    eb.cap = std::max<int64_t>(nb, 1);
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const size_t nn = (size_t)B.n * B.n;
        const size_t ne = (size_t)B.n * B.eta;
        ef::ExactBlockDev& d = eb.blk[b];
        d = ef::ExactBlockDev{};
        exact_block_geometry(c, b, eb.cap, d);
        tb.S0[b] = cv.take<double2>(nn);
        tb.cols[b] = cv.take<int>(B.cols.size());
        d.S0C = cv.take<double2>(ne);
        d.T = cv.take<double2>((size_t)B.L * nn);
        d.F = cv.take<uint32_t>(B.F.size());
        eb.Omega[b] = cv.take<double2>(B.Omega.size());
        eb.Omega32[b] = cv.take<float2>(B.Omega32.size());
        eb.OmegaHat[b] = cv.take<double2>(B.OmegaHat.size());
        eb.OmegaHatFF[b] = cv.take<float4>(B.OmegaHat.size());
        eb.sh[b] = cv.take<uint32_t>(B.sh.size());
        eb.perm[b] = cv.take<uint32_t>(B.perm.size());
        eb.goff[b] = cv.take<uint32_t>(B.goff.size());
        eb.inv_off[b] = cv.take<uint32_t>(B.inv_off.size());
        eb.inv_xs[b] = cv.take<uint32_t>(B.inv_xs.size());
    }
    eb.WS = cv.take<double2>(c->WS.size());
    eb.WS32 = cv.take<float2>(c->WS32.size());
    eb.WSFF = cv.take<float4>(c->WS.size());
    for (int b = 0; b < c->nblocks; ++b) {
        HostBlock& B = c->blk[b];
        const size_t ny = (size_t)1 << B.r;
        const size_t ne = (size_t)B.n * B.eta;
        ef::ExactBlockDev& d = eb.blk[b];
        d.M64 = cv.take<double2>(ny * ne);
        d.M32 = want32 ? cv.take<float2>(ny * ne) : nullptr;
        d.ML32 = want32 ? cv.take<float2>(ny * ne) : nullptr;
        d.D32 = c->opt.precision != EF_PREC_FP64 ? cv.take<float2>(ny * (size_t)eb.cap) : nullptr;
        d.E32 = c->opt.precision != EF_PREC_FP64 ? cv.take<uint16_t>(ny * (size_t)eb.cap) : nullptr;
        d.D64 = c->opt.precision != EF_PREC_FP32_MINOR ? cv.take<double2>(ny * (size_t)eb.cap) : nullptr;
    }
    eb.list = cv.take<int>((size_t)eb.cap);
    eb.list2 = cv.take<int>((size_t)eb.cap);
    eb.count = cv.take<int>(4);
    eb.recomp = cv.take<unsigned long long>(2);
    if (per_minor_recompute(c))
        for (int b = 0; b < c->nblocks; ++b)
            eb.mlist[b] = cv.take<int2>(((size_t)1 << c->blk[b].r) * (size_t)eb.cap);
    return (cv.off + 255) & ~(size_t)255;
}

template <typename T>
cudaError_t copy_in(const T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(const_cast<T*>(dst), src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// std::complex<double> has the layout of double2 (real, imaginary)
cudaError_t copy_in_c(const double2* dst, const cd* src, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    return cudaMemcpyAsync(const_cast<double2*>(dst), src, count * sizeof(double2), cudaMemcpyHostToDevice, s);
}

}  // namespace

extern "C" int ef_prob_exact_noalloc_dev(ef_circuit* c, const uint64_t* d_bits, int64_t nb, double* d_out,
                                         double* d_err_out, void* stream) {
    if (!c) return fail(EF_EINVAL, "NULL circuit");
    if (nb < 0 || (nb > 0 && (!d_bits || !d_out))) return fail(EF_EINVAL, "bad bitstring/output arguments");
    if (nb > 2147483647ll) return fail(EF_EINVAL, "more than 2^31-1 bitstrings per call");
    if (!c->exact_ok) return fail(EF_EUNSUPPORTED, c->exact_why);
    const cudaStream_t s = (cudaStream_t)stream;
    const bool fp64_only = c->opt.precision == EF_PREC_FP64;
    ExactBuffers eb{};
    NoAllocTables tb{};
    const size_t need = noalloc_layout(c, nb, !fp64_only, nullptr, eb, tb);
    if (need > kNoAllocBytes) {
        const size_t fixed = noalloc_layout(c, 1, !fp64_only, nullptr, eb, tb);
        const size_t per = nb > 1 ? (need - fixed) / (size_t)(nb - 1) + 1 : 1;
        const int64_t fit = fixed < kNoAllocBytes ? 1 + (int64_t)((kNoAllocBytes - fixed) / per) : 0;
        return fail(EF_EINVAL, "ef_prob_exact_noalloc_dev: this call needs " + std::to_string(need) +
                                   " bytes of scratch, the fixed scratch holds " + std::to_string(kNoAllocBytes) +
                                   "; pass at most " + std::to_string(fit) + " bitstrings per call for this circuit");
    }
    unsigned char* base = nullptr;
    int rc = noalloc_base(&base);
    if (rc) return rc;
    noalloc_layout(c, nb, !fp64_only, base, eb, tb);

    if (c->has_last_stream && c->last_stream != s) EF_CK(cudaStreamSynchronize(c->last_stream));
    c->last_stream = s;
    c->has_last_stream = true;
    c->stats = ef_stats{};
    c->last_mode = 1;
    c->last_fp64_list_pending = 0;
    c->last_recomp = nullptr;
    c->timed = false;
    c->stats.logical_branch_dets = nb * (int64_t)std::ldexp(1.0, (int)c->cps.size());
    if (nb == 0) return EF_OK;

    // the tables are copied in unless this circuit, with these angles, was the
    // scratch's last user on this device
    int dev = 0;
    EF_CK(cudaGetDevice(&dev));
    bool have_tables;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        have_tables = g_noalloc_owner[dev][0] == c->uid && g_noalloc_owner[dev][1] == c->tables_gen;
        g_noalloc_owner[dev][0] = c->uid;
        g_noalloc_owner[dev][1] = c->tables_gen;
    }
    ef::LaunchStats st;
    for (int b = 0; b < c->nblocks && !have_tables; ++b) {
        HostBlock& B = c->blk[b];
        const size_t nn = (size_t)B.n * B.n;
        const ef::ExactBlockDev& d = eb.blk[b];
        EF_CK(copy_in_c(tb.S0[b], B.S.data(), nn, s));
        EF_CK(copy_in(tb.cols[b], B.cols, s));
        if (B.L > 0) EF_CK(copy_in_c(d.T, B.T.data() + nn, (size_t)B.L * nn, s));
        EF_CK(copy_in(d.F, B.F, s));
        EF_CK(copy_in_c(eb.Omega[b], B.Omega.data(), B.Omega.size(), s));
        EF_CK(copy_in(eb.Omega32[b], B.Omega32, s));
        EF_CK(copy_in_c(eb.OmegaHat[b], B.OmegaHat.data(), B.OmegaHat.size(), s));
        EF_CK(copy_in(eb.OmegaHatFF[b], B.OmegaHatFF, s));
        EF_CK(copy_in(eb.sh[b], B.sh, s));
        EF_CK(copy_in(eb.perm[b], B.perm, s));
        EF_CK(copy_in(eb.goff[b], B.goff, s));
        EF_CK(copy_in(eb.inv_off[b], B.inv_off, s));
        EF_CK(copy_in(eb.inv_xs[b], B.inv_xs, s));
        k_gather_columns<<<32, 128, 0, s>>>(tb.S0[b], tb.cols[b], B.n, B.eta, const_cast<double2*>(d.S0C));
        EF_CK(cudaGetLastError());
        st.launches += 1;
    }
    if (!have_tables) {
        EF_CK(copy_in_c(eb.WS, c->WS.data(), c->WS.size(), s));
        EF_CK(copy_in(eb.WS32, c->WS32, s));
        EF_CK(copy_in(eb.WSFF, c->WSFF, s));
    }
    const int rc2 = run_exact(c, eb, d_bits, nb, d_out, d_err_out, s, st);
    if (rc2) {  // the tables may be partly written: copy them again next time
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        g_noalloc_owner[dev][0] = 0;
    }
    return rc2;
}

// =================================================================== multi-circuit batch
//
// A batch runs many circuits of uneven size in one CUDA graph. Exact
// circuits (FP32 minors) share persistent work-queue LU kernels, one per
// particle count, whose CTAs pull (circuit block, bitstring tile, pattern
// chunk) items from a device counter; the pattern-chunk size of every queue
// is chosen on first use by timing the candidates on the batch's own data.
// Raw Estimate circuits and the per-circuit combines run on forked streams.
// The first call for a given set of arguments plans, runs the work directly
// (its results are final) and captures the graph; later calls with the same
// arguments replay it.

struct ef_batch {
    std::vector<ef_circuit*> cs;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> key;
    struct Item {
        int mode = 0;  // 1 exact via the work queues, 2 exact on its own launches, 3 Raw Estimate
        ExactBuffers eb{};
        ef::ApproxDev a{};
        const uint64_t* bits = nullptr;
        int64_t nb = 0;
        double* out = nullptr;
    };
    std::vector<Item> items;
    struct Class {
        int eta = 0;
        int first = 0, count = 0;  // entries [first, first + count)
        int64_t n_items = 0;
        size_t smem = 0;
    };
    std::vector<Class> classes;
    std::vector<ef::QueueEntry> entries;
    std::vector<std::pair<int, int>> entry_src;  // (item, block) of each entry
    DBuf dEntries, dHeads;
    std::map<int, int> tuned;  // eta -> pattern-chunk log2
    int64_t launches = 0;
    int64_t logical = 0;

    ~ef_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaStream_t s : side) cudaStreamDestroy(s);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        dEntries.release();
        dHeads.release();
    }
};

namespace {

constexpr int kBatchSide = 4;

// Fill the queue entries of class k with chunk size 2^cl (capped per entry).
void batch_layout_class(ef_batch* bt, int k, int cl) {
    ef_batch::Class& C = bt->classes[k];
    int64_t begin = 0;
    size_t smem = 0;
    for (int e = C.first; e < C.first + C.count; ++e) {
        ef::QueueEntry& E = bt->entries[e];
        const HostBlock& B = bt->cs[bt->entry_src[e].first]->blk[bt->entry_src[e].second];
        int c = std::min(cl, B.r);
        while (c > 0 && ((size_t)1 << c) * B.n * (size_t)(B.eta | 1) * sizeof(float2) > 48 * 1024) --c;
        E.blk.c_log2 = c;
        E.blk.n_chunks = 1 << (B.r - c);
        E.tiles = (E.nb + 127) / 128;
        E.item_begin = begin;
        begin += E.tiles * E.blk.n_chunks;
        smem = std::max(smem, ((size_t)1 << c) * B.n * (size_t)(B.eta | 1) * sizeof(float2));
    }
    C.n_items = begin;
    C.smem = smem;
}

int batch_upload_entries(ef_batch* bt) {
    EF_CK(bt->dEntries.ensure(std::max<size_t>(1, bt->entries.size()) * sizeof(ef::QueueEntry)));
    if (!bt->entries.empty())
        EF_CK(cudaMemcpy(bt->dEntries.p, bt->entries.data(), bt->entries.size() * sizeof(ef::QueueEntry),
                         cudaMemcpyHostToDevice));
    return EF_OK;
}

int batch_launch_queue(ef_batch* bt, int k, cudaStream_t s, ef::LaunchStats& st) {
    const ef_batch::Class& C = bt->classes[k];
    unsigned long long* head = bt->dHeads.as<unsigned long long>() + k;
    EF_CK(cudaMemsetAsync(head, 0, sizeof(unsigned long long), s));
    const ef::QueueEntry* q = bt->dEntries.as<ef::QueueEntry>() + C.first;
    EF_CK(ef::launch_queue_lu_f32(C.eta, q, C.count, C.n_items, head, C.smem, 0, s, st));
    return EF_OK;
}

// Every launch of one batch execution (direct or under capture).
int batch_enqueue(ef_batch* bt, cudaStream_t s, ef::LaunchStats& st) {
    const int ns = (int)bt->side.size();
    EF_CK(cudaEventRecord(bt->ev[0], s));
    for (int k = 0; k < ns; ++k) EF_CK(cudaStreamWaitEvent(bt->side[k], bt->ev[0], 0));
    int rr = 0;
    for (size_t i = 0; i < bt->items.size(); ++i) {
        ef_batch::Item& it = bt->items[i];
        if (it.mode != 3 || it.nb == 0) continue;
        int rc = approx_enqueue(bt->cs[i], it.a, it.bits, it.out, nullptr, nullptr, bt->side[rr++ % ns], st);
        if (rc) return rc;
    }
    for (size_t i = 0; i < bt->items.size(); ++i) {
        ef_batch::Item& it = bt->items[i];
        if ((it.mode != 1 && it.mode != 2) || it.nb == 0) continue;
        ef_circuit* c = bt->cs[i];
        int rc = exact_enqueue_build(c, it.eb, s, st);
        if (rc) return rc;
        if (c->opt.precision == EF_PREC_AUTO)
            EF_CK(cudaMemsetAsync(it.eb.recomp, 0, 2 * sizeof(unsigned long long), s));
    }
    for (size_t k = 0; k < bt->classes.size(); ++k) {
        int rc = batch_launch_queue(bt, (int)k, s, st);
        if (rc) return rc;
    }
    EF_CK(cudaEventRecord(bt->ev[1], s));
    for (int k = 0; k < ns; ++k) EF_CK(cudaStreamWaitEvent(bt->side[k], bt->ev[1], 0));
    for (size_t i = 0; i < bt->items.size(); ++i) {
        ef_batch::Item& it = bt->items[i];
        if ((it.mode != 1 && it.mode != 2) || it.nb == 0) continue;
        ef_circuit* c = bt->cs[i];
        cudaStream_t ss = bt->side[rr++ % ns];
        const ef::ExactCombineDev cm = make_combine(c, it.eb);
        if (it.mode == 1) {
            int rc = exact_enqueue_combine(c, it.eb, cm, it.bits, it.nb, it.out, nullptr, ss, st);
            if (rc) return rc;
            continue;
        }
        // circuits outside the work queues: their own launches, slice by slice
        for (int64_t off = 0; off < it.nb; off += it.eb.cap) {
            const int64_t nbb = std::min(it.eb.cap, it.nb - off);
            int rc = exact_enqueue_lu(c, it.eb, it.bits + 2 * off, nbb, ss, st);
            if (rc) return rc;
            rc = exact_enqueue_combine(c, it.eb, cm, it.bits + 2 * off, nbb, it.out + off, nullptr, ss, st);
            if (rc) return rc;
        }
    }
    for (int k = 0; k < ns; ++k) {
        EF_CK(cudaEventRecord(bt->ev[2 + k], bt->side[k]));
        EF_CK(cudaStreamWaitEvent(s, bt->ev[2 + k], 0));
    }
    return EF_OK;
}

// Time each candidate pattern-chunk size of class k on the batch's data.
int batch_autotune(ef_batch* bt, int k, cudaStream_t s) {
    const int eta = bt->classes[k].eta;
    auto it = bt->tuned.find(eta);
    if (it != bt->tuned.end()) {
        batch_layout_class(bt, k, it->second);
        return EF_OK;
    }
    cudaEvent_t e0, e1;
    EF_CK(cudaEventCreate(&e0));
    EF_CK(cudaEventCreate(&e1));
    int best_c = 0;
    float best_ms = 1e30f;
    for (int cl = 1; cl <= 5; ++cl) {
        batch_layout_class(bt, k, cl);
        int rc = batch_upload_entries(bt);
        if (rc) return rc;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            ef::LaunchStats st;
            EF_CK(cudaEventRecord(e0, s));
            rc = batch_launch_queue(bt, k, s, st);
            if (rc) return rc;
            EF_CK(cudaEventRecord(e1, s));
            EF_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            EF_CK(cudaEventElapsedTime(&ms, e0, e1));
            ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best_c = cl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt->tuned[eta] = best_c;
    batch_layout_class(bt, k, best_c);
    return EF_OK;
}

}  // namespace

extern "C" int ef_batch_create(ef_circuit* const* cs, int32_t nc, ef_batch** out) {
    if (!out) return fail(EF_EINVAL, "out is NULL");
    *out = nullptr;
    if (nc <= 0 || !cs) return fail(EF_EINVAL, "a batch needs at least one circuit");
    for (int i = 0; i < nc; ++i) {
        if (!cs[i]) return fail(EF_EINVAL, "NULL circuit in batch");
        // a circuit's workspace holds one call's branch matrices, determinants
        // and partial sums, so two entries of one circuit would overwrite each other
        for (int j = 0; j < i; ++j)
            if (cs[j] == cs[i])
                return fail(EF_EINVAL, "circuit " + std::to_string(i) + " appears twice in the batch (entry " +
                                           std::to_string(j) + "); create a second circuit for it");
    }
    ef_batch* bt = new (std::nothrow) ef_batch();
    if (!bt) return fail(EF_ENOMEM, "host allocation failed");
    bt->cs.assign(cs, cs + nc);
    cudaError_t e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
    for (int k = 0; k < kBatchSide && e == cudaSuccess; ++k) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) bt->side.push_back(s);
    }
    for (int k = 0; k < 2 + kBatchSide && e == cudaSuccess; ++k) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) bt->ev.push_back(ev);
    }
    if (e == cudaSuccess) e = bt->dHeads.ensure(64 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        delete bt;
        return fail(EF_ECUDA, std::string("ef_batch_create: ") + cudaGetErrorString(e));
    }
    *out = bt;
    return EF_OK;
}

extern "C" int ef_batch_destroy(ef_batch* bt) {
    if (!bt) return EF_OK;
    if (bt->cap) cudaStreamSynchronize(bt->cap);
    for (cudaStream_t s : bt->side) cudaStreamSynchronize(s);
    delete bt;
    return EF_OK;
}

extern "C" int ef_batch_prob_dev(ef_batch* bt, const uint64_t* const* d_bits, const int64_t* nb,
                                 double* const* d_out, const int64_t* n_traj, uint64_t seed, void* stream) {
    if (!bt) return fail(EF_EINVAL, "NULL batch");
    if (!d_bits || !nb || !d_out || !n_traj) return fail(EF_EINVAL, "NULL argument array");
    const cudaStream_t s = (cudaStream_t)stream;
    const int nc = (int)bt->cs.size();
    std::vector<uint64_t> key = {seed};
    bool dirty = false;
    for (int i = 0; i < nc; ++i) {
        if (nb[i] < 0 || (nb[i] > 0 && (!d_bits[i] || !d_out[i])) || n_traj[i] < 0)
            return fail(EF_EINVAL, "bad arguments for circuit " + std::to_string(i));
        key.insert(key.end(), {(uint64_t)(uintptr_t)d_bits[i], (uint64_t)nb[i], (uint64_t)(uintptr_t)d_out[i],
                               (uint64_t)n_traj[i], (uint64_t)bt->cs[i]->opt.precision});
        dirty = dirty || bt->cs[i]->dirty;
    }
    // the graph holds addresses of the circuits' workspaces: a call outside the
    // batch that regrew one of them (its epoch moved) forces a new plan
    std::vector<uint64_t> key_now = key;
    for (int i = 0; i < nc; ++i) key_now.push_back(bt->cs[i]->ws_epoch);
    if (bt->exec && key_now == bt->key && !dirty) {
        EF_CK(cudaGraphLaunch(bt->exec, s));
        return EF_OK;
    }
    if (bt->exec) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    if (bt->graph) {
        cudaGraphDestroy(bt->graph);
        bt->graph = nullptr;
    }
    // plan: tables uploaded, buffers sized, modes chosen
    bt->items.assign(nc, ef_batch::Item{});
    bt->logical = 0;
    for (int i = 0; i < nc; ++i) {
        ef_circuit* c = bt->cs[i];
        ef_batch::Item& it = bt->items[i];
        it.bits = d_bits[i];
        it.nb = nb[i];
        it.out = d_out[i];
        int rc;
        if (n_traj[i] == 0) {
            if (!c->exact_ok) return fail(EF_EUNSUPPORTED, "circuit " + std::to_string(i) + ": " + c->exact_why);
            rc = begin_call(c, s, 1);
            if (rc) return rc;
            const int64_t cap = exact_batch(c, std::max<int64_t>(nb[i], 1), (size_t)2 << 30);
            rc = exact_buffers(c, cap, it.eb);
            if (rc) return rc;
            bool q = cap >= nb[i] && c->opt.precision != EF_PREC_FP64;
            for (int b = 0; b < c->nblocks; ++b) q = q && c->blk[b].eta <= ef::kMaxEtaThread;
            it.mode = q ? 1 : 2;
            bt->logical += nb[i] * (int64_t)std::ldexp(1.0, (int)c->cps.size());
        } else {
            rc = begin_call(c, s, 2);
            if (rc) return rc;
            rc = approx_setup(c, nb[i], n_traj[i], seed, 0, it.a);
            if (rc) return rc;
            it.mode = 3;
            bt->logical += nb[i] * n_traj[i];
        }
    }
    EF_CK(cudaStreamSynchronize(s));
    // work-queue classes by particle count
    bt->classes.clear();
    bt->entries.clear();
    bt->entry_src.clear();
    std::map<int, std::vector<std::pair<int, int>>> by_eta;
    for (int i = 0; i < nc; ++i)
        if (bt->items[i].mode == 1 && bt->items[i].nb > 0)
            for (int b = 0; b < bt->cs[i]->nblocks; ++b) by_eta[bt->cs[i]->blk[b].eta].push_back({i, b});
    if ((int)by_eta.size() > 64) return fail(EF_EUNSUPPORTED, "more than 64 particle-count classes");
    for (auto& kv : by_eta) {
        ef_batch::Class C;
        C.eta = kv.first;
        C.first = (int)bt->entries.size();
        // larger pieces first: fewer stragglers at the end of the queue
        std::vector<std::pair<int, int>> src = kv.second;
        std::stable_sort(src.begin(), src.end(), [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
            const double wx = (double)bt->items[x.first].nb * std::ldexp(1.0, bt->cs[x.first]->blk[x.second].r);
            const double wy = (double)bt->items[y.first].nb * std::ldexp(1.0, bt->cs[y.first]->blk[y.second].r);
            return wx > wy;
        });
        for (auto& pr : src) {
            ef::QueueEntry E{};
            E.blk = bt->items[pr.first].eb.blk[pr.second];
            E.bits = bt->items[pr.first].bits;
            E.nb = bt->items[pr.first].nb;
            bt->entries.push_back(E);
            bt->entry_src.push_back(pr);
        }
        C.count = (int)bt->entries.size() - C.first;
        bt->classes.push_back(C);
    }
    // branch matrices first (the autotuner times real work), then tune, then run
    ef::LaunchStats st0;
    for (int i = 0; i < nc; ++i)
        if (bt->items[i].mode == 1 && bt->items[i].nb > 0) {
            int rc = exact_enqueue_build(bt->cs[i], bt->items[i].eb, s, st0);
            if (rc) return rc;
        }
    for (size_t k = 0; k < bt->classes.size(); ++k) {
        int rc = batch_autotune(bt, (int)k, s);
        if (rc) return rc;
    }
    int rc = batch_upload_entries(bt);
    if (rc) return rc;
    ef::LaunchStats st;
    rc = batch_enqueue(bt, s, st);
    if (rc) return rc;
    bt->launches = st.launches;
    // capture the same work for later calls
    EF_CK(cudaStreamSynchronize(s));
    EF_CK(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeRelaxed));
    ef::LaunchStats stc;
    rc = batch_enqueue(bt, bt->cap, stc);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(EF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    bt->graph = g;
    EF_CK(cudaGraphInstantiate(&bt->exec, bt->graph, 0));
    for (int i = 0; i < nc; ++i) key.push_back(bt->cs[i]->ws_epoch);
    bt->key = key;
    return EF_OK;
}

extern "C" int ef_batch_get_stats(ef_batch* bt, ef_stats* st) {
    if (!bt || !st) return fail(EF_EINVAL, "NULL argument");
    *st = ef_stats{};
    st->kernel_launches = bt->launches;
    st->logical_branch_dets = bt->logical;
    return EF_OK;
}
