"""GPU adjoint (ef_prob_grad, FP64) against the oracle's forward-mode
derivative and against central finite differences.

Criteria: against the oracle, |g - g_ref| <= 1e-9 * max(1, |g_ref|_inf)
(both FP64, different arithmetic orders); against central differences of
the GPU FP64 forward pass (h = 1e-6),
|g . v - FD| <= 1e-6 * max(1, |g|_inf |v|_1)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from _support import mixed_settled_circuit, neutral_gates_circuit

pytestmark = pytest.mark.gpu


def gpu_grad(lib, c, bits, g):
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_FP64)
    try:
        return lib.ef_prob_grad(h, bits, g)
    finally:
        lib.ef_circuit_destroy(h)


SMALL = [
    ("brick8_exact", lambda: W.brick8_exact()),
    ("random-n8-eta3-k5", lambda: (W.random_fig4_circuit(8, 3, 5, 2, seed=21), W.sector_bitstrings_all(8, 3))),
    ("random-n10-eta4-k6-sparse", lambda: (W.random_fig4_circuit(10, 4, 6, 1, seed=23, angle_std=2.0),
                                           W.sector_bitstrings_all(10, 4)[:80])),
    ("lucj-8q-2layer", lambda: (W.lucj_circuit(4, 2, 2, 2, n_onsite=2, n_same=1, angle_sampler=W.normal_var(0.5),
                                               seed=13), W.spin_sector_bitstrings_all(4, 2, 2))),
    ("lucj-10q-1layer", lambda: (W.lucj_circuit(5, 2, 3, 1, n_onsite=3, n_same=2, angle_sampler=W.normal_var(0.3),
                                                seed=14), W.spin_sector_bitstrings_all(5, 2, 3))),
]


@pytest.mark.parametrize("name,maker", SMALL, ids=[s[0] for s in SMALL])
def test_grad_matches_oracle_all_angles(lib, name, maker):
    c, bits = maker()
    rng = np.random.default_rng(7)
    g = rng.uniform(-1, 1, len(bits))
    p, grad = gpu_grad(lib, c, bits, g)
    ref = O.prob_gradient(c, bits, g)
    assert np.max(np.abs(grad - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(p - O.exact_probabilities(c, bits))) < 1e-12


def test_grad_edge_cases(lib):
    c, bits = W.brick8_exact()
    na = len(O.get_angles(c.gates))
    p, grad = gpu_grad(lib, c, np.zeros((0, 2), dtype=np.uint64), np.zeros(0))
    assert len(p) == 0 and np.all(grad == 0) and len(grad) == na
    # wrong-weight bitstrings contribute nothing
    bad = np.array([W.modes_to_bits([0, 1, 2])], dtype=np.uint64)
    p, grad = gpu_grad(lib, c, bad, np.ones(1))
    assert p[0] == 0 and np.all(grad == 0)


def _log_weights(p, w):
    return w / p


def test_grad_lucj40_grad_subset_against_oracle(lib):
    """The 40-qubit LUCJ gradient circuit (2x20 modes, 6a+6b, 2 layers, k=12) on 12 bitstrings:
    random directions and sampled components against the oracle."""
    c, bits, w = W.lucj40_grad()
    sub = bits[:12]
    p_ref = O.exact_probabilities(c, sub)
    g = w[:12] / p_ref
    p, grad = gpu_grad(lib, c, sub, g)
    assert np.max(np.abs(p - p_ref) / p_ref) < 1e-10
    rng = np.random.default_rng(3)
    na = len(grad)
    scale = max(1.0, np.max(np.abs(grad)))
    for _ in range(2):
        v = rng.normal(size=na)
        dref = O.prob_directional_derivative(c, sub, g, v)
        assert abs(np.dot(grad, v) - dref) <= 1e-9 * scale * np.sum(np.abs(v))
    idx = rng.choice(na, 6, replace=False).tolist() + [na - 1]
    ref = O.prob_gradient(c, sub, g, angle_indices=idx)
    assert np.max(np.abs(grad[idx] - ref)) <= 1e-9 * scale


def test_grad_lucj40_grad_full_against_finite_differences(lib):
    """All 4096 bitstrings, L = sum_b w_b log p_b, adjoint against central
    differences (h = 1e-6) of the GPU FP64 forward pass."""
    c, bits, w = W.lucj40_grad()
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_FP64)
    try:
        p = lib.ef_prob_exact(h, bits)
        ang = lib.ef_circuit_get_angles(h)
        _, grad = lib.ef_prob_grad(h, bits, w / p)

        def L(a):
            lib.ef_circuit_set_angles(h, a)
            return float(np.dot(w, np.log(lib.ef_prob_exact(h, bits))))

        rng = np.random.default_rng(11)
        hstep = 1e-6
        scale = max(1.0, np.max(np.abs(grad)))
        dirs = [rng.normal(size=len(ang)) for _ in range(2)]
        for j in rng.choice(len(ang), 4, replace=False):
            e = np.zeros(len(ang))
            e[j] = 1.0
            dirs.append(e)
        for v in dirs:
            fd = (L(ang + hstep * v) - L(ang - hstep * v)) / (2 * hstep)
            assert abs(np.dot(grad, v) - fd) <= 1e-6 * scale * np.sum(np.abs(v)), (np.dot(grad, v), fd)
    finally:
        lib.ef_circuit_destroy(h)


def test_autograd_function(lib):
    torch = pytest.importorskip("torch")
    from paper_2511_12416_gb300.autograd import BornProbabilities
    c, bits = W.lucj_circuit(4, 2, 2, 2, n_onsite=2, n_same=1, angle_sampler=W.normal_var(0.5), seed=13), \
        W.spin_sector_bitstrings_all(4, 2, 2)
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_FP64)
    try:
        ang = torch.tensor(O.get_angles(c.gates), dtype=torch.float64, requires_grad=True)
        dbits = torch.from_numpy(bits.view(np.int64)).cuda()
        wts = torch.linspace(0.1, 1.0, len(bits), dtype=torch.float64, device="cuda")
        p = BornProbabilities.apply(ang, h, dbits)
        loss = (wts * torch.log(p)).sum()
        loss.backward()
        g_ref = O.prob_gradient(c, bits, (wts / p).detach().cpu().numpy())
        assert np.max(np.abs(ang.grad.numpy() - g_ref)) <= 1e-9 * max(1.0, np.max(np.abs(g_ref)))
    finally:
        lib.ef_circuit_destroy(h)



def test_grad_with_probability_neutral_gates(lib):
    """The Exact path leaves controlled-phase gates that no rotation touches
    before or after out of its enumeration (each multiplies every amplitude by
    a unit-modulus factor). The adjoint must still match the oracle, which keeps
    every gate, with a zero gradient for those gates' angles."""
    c, neutral, active = neutral_gates_circuit()
    bits = W.sector_bitstrings_all(8, 4)
    g = np.random.default_rng(8).uniform(-1, 1, len(bits))
    p, grad = gpu_grad(lib, c, bits, g)
    ref = O.prob_gradient(c, bits, g)
    assert np.max(np.abs(grad - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(p - O.exact_probabilities(c, bits))) < 1e-12
    assert abs(ref[active]) > 1e-3 and abs(grad[active]) > 1e-3
    assert np.all(np.abs(ref[neutral]) < 1e-12) and np.all(np.abs(grad[neutral]) < 1e-12)


def test_mixed_settled_gate_exact_and_gradient(lib):
    """A controlled phase whose one mode is untouched by rotations before it and
    whose other mode is untouched after it is left out of the Exact enumeration;
    probabilities (FP64 and EF_PREC_AUTO) and the adjoint still match the
    oracle, which keeps it, and its angle's gradient is zero."""
    c, neutral, active = mixed_settled_circuit()
    bits = W.sector_bitstrings_all(8, 4)
    p_ref = O.exact_probabilities(c, bits)
    floor = 1e-6 / 70
    for prec, tol in ((lib.EF_PREC_FP64, 1e-10), (lib.EF_PREC_AUTO, 1e-5)):
        h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=prec)
        try:
            p = lib.ef_prob_exact(h, bits)
        finally:
            lib.ef_circuit_destroy(h)
        assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, floor)) <= tol
    g = np.random.default_rng(9).uniform(-1, 1, len(bits))
    _, grad = gpu_grad(lib, c, bits, g)
    ref = O.prob_gradient(c, bits, g)
    assert np.max(np.abs(grad - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    assert abs(ref[neutral]) < 1e-12 and abs(grad[neutral]) < 1e-12
    assert abs(ref[active]) > 1e-4


def _oracle_dirderiv_chunk(args):
    c, bits, g, v = args
    return O.prob_directional_derivative(c, bits, g, v)


def test_grad_lucj40_grad_all_bitstrings_directional_against_oracle(lib):
    """The 40-qubit LUCJ gradient workload on all 4096 bitstrings: the adjoint
    along one random direction against the oracle's forward-mode derivative of
    L = sum_b w_b log p_b (oracle work split over host cores)."""
    import multiprocessing as mp
    import os
    c, bits, w = W.lucj40_grad()
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_FP64)
    try:
        p = lib.ef_prob_exact(h, bits)
        _, grad = lib.ef_prob_grad(h, bits, w / p)
    finally:
        lib.ef_circuit_destroy(h)
    v = np.random.default_rng(21).normal(size=len(grad))
    g = w / p
    ncores = max(1, min(32, len(os.sched_getaffinity(0))))
    chunks = [(c, bits[i::ncores], g[i::ncores], v) for i in range(ncores)]
    with mp.get_context("spawn").Pool(ncores) as pool:
        dref = float(sum(pool.map(_oracle_dirderiv_chunk, chunks)))
    scale = max(1.0, np.max(np.abs(grad)))
    assert abs(np.dot(grad, v) - dref) <= 1e-9 * scale * np.sum(np.abs(v)), (np.dot(grad, v), dref)
