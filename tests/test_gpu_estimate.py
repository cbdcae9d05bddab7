"""GPU Estimate driver (ef_prob_estimate, Section III-A with Eq. 6) against the
oracle's Estimate and against the exact probabilities.

* Parity: with FP64 minors the driver and the oracle take the same rounds,
  the same trajectory counts and the same trajectories, so the estimates agree
  within 1e-10 of max(p, p_floor) and the counts are equal.
* Guarantee: over many seeds and bitstrings, |p_hat - p| > eps happens at most
  with frequency delta (plus a three-sigma binomial margin); the rounds spend
  fewer trajectories than one Raw Estimate with p_max = 1."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _estimate(lib, c, bits, eps, delta, seed, precision):
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=precision)
    try:
        return lib.ef_prob_estimate(h, bits, eps, delta, seed=seed)
    finally:
        lib.ef_circuit_destroy(h)


def test_estimate_matches_oracle_estimate(lib):
    c, bits = W.brick8_exact()
    sub = bits[[2, 11, 30, 55]]
    eps, delta, seed = 0.02, 0.01, 77
    p_ref, se_ref, t_ref = O.estimate(c, sub, eps, delta, seed, b_indices=[0, 1, 2, 3])
    p, se, t = _estimate(lib, c, sub, eps, delta, seed, lib.EF_PREC_FP64)
    floor = 1e-6 / math.comb(8, 4)
    assert np.array_equal(t, t_ref)
    assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, floor)) <= 1e-10
    assert np.max(np.abs(se - se_ref) / np.maximum(se_ref, floor)) <= 1e-8


def test_estimate_matches_oracle_on_spread_outcomes_across_2_32(lib):
    """The same parity on outcomes whose probabilities run from 0.64 down to
    1.2e-4 (a 10-mode random circuit, extent 14.6), at global indices that
    cross 2^32 and with a seed that fills both key words."""
    c = W.random_fig4_circuit(10, 4, 7, 3, seed=31, angle_std=1.2)
    bits = W.sector_bitstrings_all(10, 4)
    pe = O.exact_probabilities(c, bits)
    pick = np.argsort(-pe)[[0, 3, 8, 14]]
    sub = bits[pick]
    eps, delta, seed, base = 0.05, 0.05, 0xFEDC_BA98_7654_3210, (1 << 32) - 2
    p_ref, se_ref, t_ref = O.estimate(c, sub, eps, delta, seed, b_indices=[base + i for i in range(len(sub))])
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_FP64)
    try:
        p, se, t = lib.ef_prob_estimate(h, sub, eps, delta, seed=seed, index_base=base)
    finally:
        lib.ef_circuit_destroy(h)
    floor = 1e-6 / math.comb(10, 4)
    assert np.array_equal(t, t_ref)
    assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, floor)) <= 1e-10
    assert np.max(np.abs(se - se_ref) / np.maximum(se_ref, floor)) <= 1e-8
    assert np.all(np.abs(p - pe[pick]) <= eps)


@pytest.mark.parametrize("prec", ["fp64", "auto"])
def test_estimate_guarantee_over_seeds(lib, prec):
    c = W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1), seed=7)
    bits = W.spin_sector_bitstrings_all(6, 3, 3)[:60]
    p = O.exact_probabilities(c, bits)
    eps, delta = 0.01, 0.1
    precision = lib.EF_PREC_FP64 if prec == "fp64" else lib.EF_PREC_AUTO
    fails, n = 0, 0
    spent = []
    for seed in range(25):
        ph, _, t = _estimate(lib, c, bits, eps, delta, 1000 + seed, precision)
        fails += int(np.count_nonzero(np.abs(ph - p) > eps))
        n += len(bits)
        spent.append(t)
    margin = 3.0 * math.sqrt(delta * (1 - delta) / n)
    assert fails / n <= delta + margin, (fails, n)
    one_shot = O.trajectory_count_bound(eps, delta, 1.0, O.extent(c.gates))
    assert np.mean(spent) < one_shot


def test_estimate_edge_cases(lib):
    c, bits = W.brick8_exact()
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates)
    try:
        bad = np.array([W.modes_to_bits([0, 1])], dtype=np.uint64)
        p, se, t = lib.ef_prob_estimate(h, bad, 0.05, 0.1)
        assert p[0] == 0 and t[0] == 0
        p, se, t = lib.ef_prob_estimate(h, np.zeros((0, 2), dtype=np.uint64), 0.05, 0.1)
        assert len(p) == 0
        for eps, delta in ((0.0, 0.1), (0.1, 0.0), (0.1, 1.0)):
            with pytest.raises(lib.ExtraFermError):
                lib.ef_prob_estimate(h, bits[:2], eps, delta)
    finally:
        lib.ef_circuit_destroy(h)
