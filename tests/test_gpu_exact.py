"""GPU parity of the Exact algorithm (Eqs. 8-9) against the FP64 CPU oracle.

Tolerances (element by element, on the same seeded inputs):
  * FP64 path: |p_gpu - p| <= 1e-10 * max(p, p_floor);
  * FP32 minors with FP64 fallback (EF_PREC_AUTO): <= 1e-5 * max(p, p_floor);
  * FP32 minors alone: the library's own per-result error estimate must bound
    the observed error;
with p_floor = 1e-6 / |sector| (|sector| = number of bitstrings with the
initial state's per-block Hamming weights)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from _support import likely_bitstrings, neutral_gates_circuit

pytestmark = pytest.mark.gpu


def sector_size(c):
    meta = c.meta
    if "norb" in meta:
        return math.comb(meta["norb"], meta["n_alpha"]) * math.comb(meta["norb"], meta["n_beta"])
    return math.comb(c.n_modes, len(c.occupied_modes()))


def rel_err(p_gpu, p_ref, floor):
    return np.abs(p_gpu - p_ref) / np.maximum(p_ref, floor)


def run_exact(lib, c, bits, precision, want_err=False, **kw):
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=precision, **kw)
    try:
        res = lib.ef_prob_exact(h, bits, want_err=want_err)
        st = lib.ef_circuit_get_stats(h)
    finally:
        lib.ef_circuit_destroy(h)
    return res, st


def _shallow26():
    c = W.uneven_batch64(7)[6][0]
    return c, likely_bitstrings(c, 200, 9)


SMALL = [
    ("brick8_exact", lambda: W.brick8_exact()),
    ("brick-after", lambda: (W.brick_circuit(8, 4, 3, seed=0, cphase_between=False), W.sector_bitstrings_all(8, 4))),
    ("random-n10-eta5-k6", lambda: (W.random_fig4_circuit(10, 5, 6, 3, seed=22), W.sector_bitstrings_all(10, 5))),
    ("random-n12-eta1-k4", lambda: (W.random_fig4_circuit(12, 1, 4, 2, seed=24), W.sector_bitstrings_all(12, 1))),
    ("random-n12-eta11-k5", lambda: (W.random_fig4_circuit(12, 11, 5, 2, seed=25), W.sector_bitstrings_all(12, 11))),
    ("random-n14-eta7-k9", lambda: (W.random_fig4_circuit(14, 7, 9, 3, seed=26, angle_std=2.0),
                                    W.sector_bitstrings(14, 7, 300, np.random.default_rng(3)))),
    ("lucj-12q", lambda: (W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1, math.pi),
                                         seed=7), W.spin_sector_bitstrings_all(6, 3, 3))),
    ("lucj-10q-2layer", lambda: (W.lucj_circuit(5, 2, 2, 2, n_onsite=3, n_same=2, angle_sampler=W.normal_var(0.5),
                                                seed=8), W.spin_sector_bitstrings_all(5, 2, 2))),
    ("lucj-20q-uneven", lambda: (W.lucj_circuit(10, 4, 2, 1, n_onsite=5, n_same=3, angle_sampler=W.normal_var(0.3),
                                                seed=9), W.spin_sector_bitstrings(10, 4, 2, 517, np.random.default_rng(4)))),
    # 26 modes, 7+7 particles, one brick layer: the last rows of every branch
    # matrix are exactly zero, so the exchange form's coefficients carry FP64
    # rounding noise where the exact values vanish (tiny FP32 pivots)
    ("shallow-26q-zero-rows", lambda: _shallow26()),
]


@pytest.mark.parametrize("name,maker", SMALL, ids=[s[0] for s in SMALL])
def test_exact_fp64_matches_oracle(lib, name, maker):
    c, bits = maker()
    p_ref = O.exact_probabilities(c, bits)
    p, st = run_exact(lib, c, bits, lib.EF_PREC_FP64)
    floor = 1e-6 / sector_size(c)
    assert np.max(rel_err(p, p_ref, floor)) <= 1e-10
    assert st["logical_branch_dets"] == len(bits) * 2 ** c.n_cphase


@pytest.mark.parametrize("name,maker", SMALL, ids=[s[0] for s in SMALL])
def test_exact_auto_matches_oracle_within_1e5(lib, name, maker):
    c, bits = maker()
    p_ref = O.exact_probabilities(c, bits)
    (p, err), st = run_exact(lib, c, bits, lib.EF_PREC_AUTO, want_err=True)
    floor = 1e-6 / sector_size(c)
    assert np.max(rel_err(p, p_ref, floor)) <= 1e-5


@pytest.mark.parametrize("name,maker", SMALL, ids=[s[0] for s in SMALL])
def test_exact_fp32_error_estimate_bounds_error(lib, name, maker):
    c, bits = maker()
    p_ref = O.exact_probabilities(c, bits)
    (p, err), _ = run_exact(lib, c, bits, lib.EF_PREC_FP32_MINOR, want_err=True)
    floor = 1e-6 / sector_size(c)
    actual = rel_err(p, p_ref, floor)
    # the estimate bounds every error that is not negligible next to the 1e-5 bar
    assert np.all(actual <= np.maximum(err, 1e-8)), (actual / np.maximum(err, 1e-300)).max()


def test_exact_edge_cases(lib):
    c, bits = W.brick8_exact()
    # wrong Hamming weight -> exactly 0; empty call; ragged count
    bad = np.array([W.modes_to_bits([0, 1, 2]), W.modes_to_bits([0, 1, 2, 3, 4]), W.modes_to_bits([])],
                   dtype=np.uint64)
    for prec in (lib.EF_PREC_FP64, lib.EF_PREC_FP32_MINOR, lib.EF_PREC_AUTO):
        p, _ = run_exact(lib, c, bad, prec)
        assert np.all(p == 0.0)
        p, st = run_exact(lib, c, np.zeros((0, 2), dtype=np.uint64), prec)
        assert len(p) == 0
    # a bit at or above n_modes is an error, not a zero
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates)
    try:
        with pytest.raises(lib.ExtraFermError) as e:
            lib.ef_prob_exact(h, np.array([W.modes_to_bits([0, 1, 2, 9])], dtype=np.uint64))
        assert e.value.status == lib.EF_EINVAL
    finally:
        lib.ef_circuit_destroy(h)


def test_host_calls_leave_outputs_untouched_on_out_of_range_bits(lib):
    """A bitstring with a bit at or above n_modes makes the host-pointer calls
    return EF_EINVAL and leaves every output array as it was (the range check
    runs while the GPU works; nothing is copied back)."""
    import ctypes
    c, bits = W.brick8_exact()
    b = np.ascontiguousarray(np.concatenate([bits[:5], np.array([W.modes_to_bits([0, 1, 2, 9])],
                                                                dtype=np.uint64)]))
    L = lib.load()
    dp = ctypes.POINTER(ctypes.c_double)
    bp = b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO)
    try:
        out, err, se = (np.full(len(b), 7.0) for _ in range(3))
        rc = L.ef_prob_exact(h, bp, len(b), out.ctypes.data_as(dp), err.ctypes.data_as(dp))
        assert rc == lib.EF_EINVAL
        assert np.all(out == 7.0) and np.all(err == 7.0)
        rc = L.ef_prob_approx(h, bp, len(b), 64, 3, 0, out.ctypes.data_as(dp), se.ctypes.data_as(dp),
                              err.ctypes.data_as(dp))
        assert rc == lib.EF_EINVAL
        assert np.all(out == 7.0) and np.all(se == 7.0) and np.all(err == 7.0)
        # the circuit stays usable
        p = lib.ef_prob_exact(h, bits[:5])
        assert np.max(np.abs(p - O.exact_probabilities(c, bits[:5]))) <= 1e-5
    finally:
        lib.ef_circuit_destroy(h)


def test_exact_wrong_spin_sector_is_zero(lib):
    c = W.lucj_circuit(5, 2, 2, 1, n_onsite=3, n_same=2, angle_sampler=W.normal_var(0.5), seed=8)
    bits = np.array([W.modes_to_bits([0, 1, 2, 5]), W.modes_to_bits([0, 5, 6, 7])], dtype=np.uint64)
    p, _ = run_exact(lib, c, bits, lib.EF_PREC_AUTO)
    assert np.all(p == 0.0)
    assert np.all(O.exact_probabilities(c, bits) < 1e-30)


def test_exact_no_cphase_and_all_zero_angles(lib):
    rng = np.random.default_rng(5)
    V = W.haar_unitary(9, rng)
    c = W.Circuit(9, W.modes_to_bits([0, 2, 3, 7]), W.make_gates(W.givens_network(V)))
    bits = W.sector_bitstrings_all(9, 4)
    p, _ = run_exact(lib, c, bits, lib.EF_PREC_FP64)
    ref = np.array([abs(np.linalg.det(V[np.ix_(W.bits_to_modes(b), [0, 2, 3, 7])])) ** 2 for b in bits])
    assert np.max(np.abs(p - ref)) < 1e-13
    assert abs(p.sum() - 1.0) < 1e-12


def test_exact_sector_sums_to_one_all_precisions(lib):
    c = W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1, math.pi), seed=7)
    bits = W.spin_sector_bitstrings_all(6, 3, 3)
    for prec, tol in ((lib.EF_PREC_FP64, 1e-12), (lib.EF_PREC_AUTO, 1e-6)):
        p, _ = run_exact(lib, c, bits, prec)
        assert abs(p.sum() - 1.0) < tol


def test_exact_lucj32_exact_full_size_sampled(lib):
    """10^4 bitstrings in the bench's launch configuration; the oracle checks
    a sample (first, last and random positions) and the FP64 path checks all."""
    c, bits = W.lucj32_exact()
    floor = 1e-6 / sector_size(c)
    (p_auto, err), st = run_exact(lib, c, bits, lib.EF_PREC_AUTO, want_err=True)
    p64, _ = run_exact(lib, c, bits, lib.EF_PREC_FP64)
    assert np.max(rel_err(p_auto, p64, floor)) <= 1e-5
    rng = np.random.default_rng(77)
    idx = np.unique(np.concatenate([[0, len(bits) - 1], rng.choice(len(bits), 6, replace=False)]))
    p_ref = O.exact_probabilities(c, bits[idx])
    assert np.max(rel_err(p64[idx], p_ref, floor)) <= 1e-10
    assert np.max(rel_err(p_auto[idx], p_ref, floor)) <= 1e-5
    assert st["logical_branch_dets"] == len(bits) * 2 ** 16


@pytest.mark.parametrize("which", ["lucj32_exact", "lucj40_grad"])
def test_exact_fp32_estimate_on_full_size_workloads(lib, which):
    """At full size the FP32 path's estimate bounds its error against the
    (oracle-checked) FP64 path, and EF_PREC_AUTO meets 1e-5 everywhere."""
    c, bits = W.lucj32_exact() if which == "lucj32_exact" else W.lucj40_grad()[:2]
    floor = 1e-6 / sector_size(c)
    p64, _ = run_exact(lib, c, bits, lib.EF_PREC_FP64)
    (p32, err), _ = run_exact(lib, c, bits, lib.EF_PREC_FP32_MINOR, want_err=True)
    actual = rel_err(p32, p64, floor)
    assert np.all(actual <= np.maximum(err, 1e-8))
    (pa, _), st = run_exact(lib, c, bits, lib.EF_PREC_AUTO, want_err=True)
    assert np.max(rel_err(pa, p64, floor)) <= 1e-5
    assert st["fp64_recomputed"] < 0.2 * len(bits)


def test_exact_repeatable_and_device_api(lib):
    torch = pytest.importorskip("torch")
    c, bits = W.lucj32_exact(1000)
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO)
    try:
        p_host = lib.ef_prob_exact(h, bits)
        d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
        d_out = torch.empty(len(bits), dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        lib.ef_prob_exact_dev(h, d_bits.data_ptr(), len(bits), d_out.data_ptr(), 0, s.cuda_stream)
        s.synchronize()
        assert np.array_equal(d_out.cpu().numpy(), p_host)
        assert np.array_equal(lib.ef_prob_exact(h, bits), p_host)
    finally:
        lib.ef_circuit_destroy(h)


def test_exact_leaves_probability_neutral_gates_out(lib):
    """Of the circuit's four controlled-phase gates only the one between
    rotation layers can change a probability: the FP64 path factors 2 minors
    per bitstring (one flip bit), not 2^4, and still matches the oracle, which
    enumerates every gate."""
    c, _, _ = neutral_gates_circuit()
    bits = W.sector_bitstrings_all(8, 4)
    p, st = run_exact(lib, c, bits, lib.EF_PREC_FP64)
    assert np.max(rel_err(p, O.exact_probabilities(c, bits), 1e-6 / sector_size(c))) <= 1e-10
    assert st["executed_minor_lus"] == 2 * len(bits)
    assert st["logical_branch_dets"] == len(bits) * 2 ** 4


def test_exact_auto_tight_tolerance_float_pair_redo(lib):
    """EF_PREC_AUTO at tol = 1e-9 on 2000 bitstrings of the 32-qubit LUCJ
    workload: most results need the redo, so many determinants go through the
    float-pair warp-row LU (about 48 bits) and some results through the
    whole-bitstring FP64 redo; every result must stay within 1e-9 of the FP64
    path (pinned to the oracle by the tests above)."""
    c, bits = W.lucj32_exact(2000)
    floor = 1e-6 / sector_size(c)
    p64, _ = run_exact(lib, c, bits, lib.EF_PREC_FP64)
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO, tol=1e-9)
    try:
        p, err = lib.ef_prob_exact(h, bits, want_err=True)
        st = lib.ef_circuit_get_stats(h)
    finally:
        lib.ef_circuit_destroy(h)
    assert np.max(rel_err(p, p64, floor)) <= 1e-9
    assert st["fp64_recomputed"] > len(bits) // 2
    assert st["fp64_recomputed"] == np.count_nonzero(err < 0)
