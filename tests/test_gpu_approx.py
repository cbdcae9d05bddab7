"""GPU parity of the Raw Estimate (Eqs. 10-12) against the FP64 CPU oracle.

Both sides draw the same trajectories (Philox4x32-10 keyed by seed, global
bitstring index and trajectory number, integer thresholds), so the estimator
itself is a deterministic function compared element by element:

  * FP64 path: |p_gpu - p_oracle| <= 1e-10 * max(p, p_floor);
  * EF_PREC_AUTO (FP32 minors, FP64 recompute of the results whose estimated
    error exceeds 1e-5): |p_gpu - p_oracle| <= 1e-5 * max(p, p_floor);
  * EF_PREC_FP32_MINOR alone: the per-result error estimate bounds the
    observed error, and the error is within 1e-5 of M^2 (M = mean |Y_i|, the
    size of the Eq. 11 terms whose FP32 rounding it is).

The total number of sampled flips must match exactly."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def run_approx(lib, c, bits, t, seed, precision, index_base=0, want_err=False):
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=precision)
    try:
        p, se, err = lib.ef_prob_approx(h, bits, t, seed=seed, index_base=index_base, want_err=True)
        st = lib.ef_circuit_get_stats(h)
    finally:
        lib.ef_circuit_destroy(h)
    return (p, se, st, err) if want_err else (p, se, st)


CASES = [
    ("brick8_exact", lambda: W.brick8_exact(), 3000),
    ("random-n10-eta4-k7", lambda: (W.random_fig4_circuit(10, 4, 7, 3, seed=31, angle_std=1.2),
                                    W.sector_bitstrings_all(10, 4)[:60]), 1000),
    ("lucj-12q", lambda: (W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1),
                                         seed=7), W.spin_sector_bitstrings_all(6, 3, 3)[:50]), 2000),
    ("lucj-16q-3layer", lambda: (W.lucj_circuit(8, 3, 2, 3, n_onsite=4, n_same=2, angle_sampler=W.normal_var(0.4),
                                                seed=12), W.spin_sector_bitstrings(8, 3, 2, 40, np.random.default_rng(2))),
     2500),
]


@pytest.mark.parametrize("name,maker,t", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "auto"])
def test_approx_matches_oracle_same_trajectories(lib, name, maker, t, prec):
    c, bits = maker()
    seed = 0x1234_5678_9ABC
    p_ref, se_ref, _, flips_ref, scale = O.raw_estimate(c, bits, t=t, seed=seed, return_details=True,
                                                         return_scale=True)
    precision = {"fp64": lib.EF_PREC_FP64, "fp32": lib.EF_PREC_FP32_MINOR, "auto": lib.EF_PREC_AUTO}[prec]
    p, se, st, err = run_approx(lib, c, bits, t, seed, precision, want_err=True)
    n = c.n_modes
    floor = 1e-6 / math.comb(n, len(c.occupied_modes()))
    rel = np.abs(p - p_ref) / np.maximum(p_ref, floor)
    if prec == "fp64":
        assert np.max(rel) <= 1e-10
        assert np.all(err == 0)
    elif prec == "auto":
        assert np.max(rel) <= 1e-5, (np.max(rel), np.count_nonzero(err < 0))
        assert st["fp64_recomputed"] == np.count_nonzero(err < 0)
        assert np.all(np.abs(err[err < 0]) > 1e-5) and np.all(err[err >= 0] <= 1e-5)
    else:
        assert np.max(np.abs(p - p_ref) / np.maximum(scale * scale, floor)) <= 1e-5
        # the estimate bounds the observed error (beyond FP64 noise of the reference)
        assert np.all(rel <= err + 1e-9), (np.max(rel / np.maximum(err, 1e-30)), np.max(rel))
    assert np.max(np.abs(se - se_ref) / np.maximum(se_ref, floor)) <= (1e-8 if prec == "fp64" else 1e-3)
    assert st["sampled_flips"] == flips_ref
    assert st["logical_branch_dets"] == len(bits) * t


def test_approx_global_index_and_subsets(lib):
    """A subset called with its global index base draws the same trajectories
    as in the full call (equal within FP64 rounding of the sums; different
    trajectories would differ by far more)."""
    c = W.random_fig4_circuit(10, 4, 7, 3, seed=31, angle_std=1.2)
    bits = W.sector_bitstrings_all(10, 4)[:60]
    p_all, se_all, _ = run_approx(lib, c, bits, 500, 7, lib.EF_PREC_FP64)
    p_sub, se_sub, _ = run_approx(lib, c, bits[30:45], 500, 7, lib.EF_PREC_FP64, index_base=30)
    assert np.count_nonzero(p_all[30:45] > 1e-6) >= 5  # not a comparison of zeros
    assert np.allclose(p_sub, p_all[30:45], rtol=1e-12, atol=0)
    assert np.allclose(se_sub, se_all[30:45], rtol=1e-10, atol=0)


def test_approx_global_indices_across_2_32(lib):
    """Global bitstring indices that cross 2^32: the high index word of the
    Philox counter reaches the trajectories as in the oracle (same
    trajectories, FP64 parity), and the indices, not the positions in the
    call, select them."""
    c = W.random_fig4_circuit(10, 4, 7, 3, seed=31, angle_std=1.2)
    bits = W.sector_bitstrings_all(10, 4)
    sub = bits[np.argsort(-O.exact_probabilities(c, bits))[:20]]  # the 20 most probable outcomes
    base = (1 << 32) - 9
    seed, t = 0x0123_4567_89AB_CDEF, 700
    idx = [base + i for i in range(len(sub))]
    p_ref, se_ref = O.raw_estimate(c, sub, t=t, seed=seed, b_indices=idx)
    floor = 1e-6 / math.comb(c.n_modes, len(c.occupied_modes()))
    for prec, tol in ((lib.EF_PREC_FP64, 1e-10), (lib.EF_PREC_AUTO, 1e-5)):
        p, se, _ = run_approx(lib, c, sub, t, seed, prec, index_base=base)
        assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, floor)) <= tol, prec
        assert np.max(np.abs(se - se_ref) / np.maximum(se_ref, floor)) <= (1e-8 if tol < 1e-9 else 1e-3), prec
    # bitstrings 9.. sit at indices 2^32 + 0.., which share their low words with indices 0..
    p_low, _, _ = run_approx(lib, c, sub[9:], t, seed, lib.EF_PREC_FP64, index_base=0)
    p_low_ref, _ = O.raw_estimate(c, sub[9:], t=t, seed=seed)
    assert np.max(np.abs(p_low - p_low_ref) / np.maximum(p_low_ref, floor)) <= 1e-10
    # ... and their trajectories differ: the GPU matched both sets, so it keeps the high word
    assert np.max(np.abs(p_low_ref - p_ref[9:]) / np.maximum(p_ref[9:], floor)) > 1e-3


def test_approx_zero_angles_is_exact(lib):
    c, bits = W.brick8_exact()
    recs = [(int(g["kind"]), int(g["p"]), int(g["q"]), 0.0 if int(g["kind"]) == W.CPHASE else float(g["theta"]),
             float(g["phi"])) for g in c.gates]
    c0 = W.Circuit(8, c.occupation, W.make_gates(recs))
    p, se, st = run_approx(lib, c0, bits, 333, 1, lib.EF_PREC_FP64)
    assert np.max(np.abs(p - O.exact_probabilities(c0, bits))) < 1e-15
    assert np.all(se < 1e-14) and st["sampled_flips"] == 0


def test_approx_edge_cases(lib):
    c, bits = W.brick8_exact()
    bad = np.array([W.modes_to_bits([0, 1]), W.modes_to_bits([0, 1, 2, 3, 4])], dtype=np.uint64)
    p, se, _ = run_approx(lib, c, bad, 100, 0, lib.EF_PREC_FP32_MINOR)
    assert np.all(p == 0) and np.all(se == 0)
    p, se, _ = run_approx(lib, c, bits[:3], 1, 0, lib.EF_PREC_FP64)
    assert np.all(se == 0)
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates)
    try:
        with pytest.raises(lib.ExtraFermError):
            lib.ef_prob_approx(h, bits[:3], 0)
    finally:
        lib.ef_circuit_destroy(h)


def test_approx_unbiased_against_exact(lib):
    """Many independent seeds: the mean of alpha-estimates' |.|^2 follows the
    exact bias formula E[p_hat] = p + (E|Y|^2 - p)/t."""
    c = W.random_fig4_circuit(6, 3, 5, 2, seed=31, angle_std=1.5)
    b = W.sector_bitstrings_all(6, 3)[7:8]
    alpha, m2 = O.expected_second_moment(c, b[0])
    p = abs(alpha) ** 2
    t = 64
    bits = np.repeat(b, 2000, axis=0)  # each row has its own global index -> independent trajectories
    ph, _, _ = run_approx(lib, c, bits, t, 99, lib.EF_PREC_FP64)
    z = (ph.mean() - (p + (m2 - p) / t)) / (ph.std(ddof=1) / math.sqrt(len(ph)))
    assert abs(z) < 4.0


def test_approx_lucj52_approx_full_trajectory_count_sampled(lib):
    """The 52-qubit LUCJ workload (k=152, t = ceil(extent/eps^2)) at full t on 256
    bitstrings under EF_PREC_AUTO: the oracle checks two of them; all 256 agree
    with the GPU's FP64 path on the same trajectories (pinned to the oracle at
    1e-10 by the smaller cases) within 1e-5 of p."""
    c, bits = W.lucj52_approx(256)
    t = W.lucj52_trajectories(O.extent(c.gates))
    p, se, st, err = run_approx(lib, c, bits, t, 0, lib.EF_PREC_AUTO, want_err=True)
    idx = [0, 201]
    p_ref, se_ref = O.raw_estimate(c, bits[idx], t=t, seed=0, b_indices=idx)
    floor = 1e-6 / (math.comb(26, 5) ** 2)
    assert np.max(np.abs(p[idx] - p_ref) / np.maximum(p_ref, floor)) <= 1e-5
    assert np.all(np.isfinite(p)) and np.all(p >= 0)
    p64, _, st64 = run_approx(lib, c, bits, t, 0, lib.EF_PREC_FP64)
    assert np.max(np.abs(p - p64) / np.maximum(p64, floor)) <= 1e-5
    assert st["sampled_flips"] == st64["sampled_flips"]


# Raw Estimate circuits of the 64-circuit uneven batch with few modes and many
# controlled-phase gates (strong cancellation between trajectories): 34 is
# n=12, 3+3 particles, k=22; 2 is n=12, k=24; 33 is n=16, k=21.
BATCH_CANCELLING = [34, 2, 33]


@pytest.mark.parametrize("ci", BATCH_CANCELLING)
def test_approx_auto_on_cancelling_batch_circuits(lib, ci):
    """EF_PREC_AUTO against the FP64 path on the same trajectories (t =
    ceil(extent 1e4)), 1500 bitstrings of each circuit, within 1e-5 of
    max(p, p_floor); FP32 minors alone: the estimate bounds the observed
    error. Every trajectory that flips a given gate or flippable pair reuses
    the same rounded ratio and K entry, so these roundings add up over the
    trajectories instead of averaging out; the kernel corrects them to first
    order. The oracle checks the FP64 path on one bitstring."""
    c, bits, mode = W.uneven_batch64()[ci]
    assert mode == "approx"
    bits = bits[:1500]
    t = int(min(math.ceil(O.extent(c.gates) * 1e4), 10 ** 6))
    p64, _, _ = run_approx(lib, c, bits, t, 7, lib.EF_PREC_FP64)
    pa, _, st, ea = run_approx(lib, c, bits, t, 7, lib.EF_PREC_AUTO, want_err=True)
    p32, _, _, e32 = run_approx(lib, c, bits, t, 7, lib.EF_PREC_FP32_MINOR, want_err=True)
    floor = 1e-6 / math.comb(c.n_modes // 2, len(c.occupied_modes()) // 2) ** 2
    den = np.maximum(p64, floor)
    assert np.max(np.abs(pa - p64) / den) <= 1e-5
    assert np.all(np.abs(p32 - p64) / den <= e32 + 1e-9)
    assert st["fp64_recomputed"] == np.count_nonzero(ea < 0)
    j = int(np.argmax(np.abs(p32 - p64) / den))
    p_ref, _ = O.raw_estimate(c, bits[j:j + 1], t=t, seed=7, b_indices=[j])
    assert abs(p64[j] - p_ref[0]) <= 1e-10 * max(p_ref[0], floor)
