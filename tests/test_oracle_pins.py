"""Pins of the FP64 CPU oracle to things other than itself: a brute-force
state vector, closed forms, the paper's worked example and printed extents,
published generator vectors and statistical properties of the estimator."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _modes_list(bits):
    return [W.bits_to_modes(b) for b in bits]


# --------------------------------------------------------------------------- generator


def test_philox_known_answer_vectors():
    for v in _load("philox4x32_10_kat.json")["vectors"]:
        c = [int(h, 16) for h in v["counter"]]
        k = [int(h, 16) for h in v["key"]]
        out = O.philox4x32_10(*c, *k)
        assert [int(o) for o in out] == [int(h, 16) for h in v["output"]]


_TRITON_PROBE = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, k0_ptr, k1_ptr):
    i = tl.arange(0, 8)
    a, b, c, d = tl.random.philox_impl(tl.load(c0_ptr + i), tl.load(c1_ptr + i), tl.load(c2_ptr + i),
                                      tl.load(c3_ptr + i), tl.load(k0_ptr + i), tl.load(k1_ptr + i), 10)
    tl.store(out_ptr + i, a); tl.store(out_ptr + 8 + i, b); tl.store(out_ptr + 16 + i, c); tl.store(out_ptr + 24 + i, d)
cols = json.loads(sys.argv[1])
t = [torch.tensor(c, dtype=torch.int64).to(torch.uint32) for c in cols]
out = torch.zeros(32, dtype=torch.uint32)
k[(1,)](out, *t)
print(json.dumps([int(v) for v in out.to(torch.int64)]))
"""


def test_philox_matches_an_independent_implementation():
    """Triton's Philox4x32 (run in its CPU interpreter) agrees word for word."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    cols = rng.integers(0, 2**32, size=(6, 8), dtype=np.uint64)
    res = subprocess.run([sys.executable, "-c", _TRITON_PROBE, json.dumps(cols.tolist())],
                         capture_output=True, text=True, timeout=300)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr.strip().splitlines()[-1][:200])
    got = np.array(json.loads(res.stdout.strip().splitlines()[-1]), dtype=np.uint64).reshape(4, 8)
    want = np.stack(O.philox4x32_10(*cols))
    assert np.array_equal(got, want)


# --------------------------------------------------------------------------- Eq. 7 / Eq. 16


def test_cphase_decomposition_identity():
    """c(theta) = e^{i theta/4}[cos(theta/4) d0 + i sin(theta/4) d1] (Eq. 7),
    also for angles outside (-pi, pi] once wrapped."""
    for theta in [0.0, 0.3, -1.2, math.pi, 2.5 * math.pi, -7.0]:
        th = O.wrap_angle(theta)
        assert -math.pi < th <= math.pi
        c = np.diag([1, 1, 1, np.exp(1j * theta)])
        d0 = np.diag([np.exp(-0.5j * th), 1, 1, np.exp(0.5j * th)])
        d1 = np.diag([np.exp(-0.5j * th), -1, -1, np.exp(0.5j * th)])
        rhs = np.exp(0.25j * th) * (math.cos(th / 4) * d0 + 1j * math.sin(th / 4) * d1)
        assert np.allclose(c, rhs, atol=1e-14)


# --------------------------------------------------------------------------- Exact vs state vector


@pytest.mark.parametrize("maker", [
    lambda: W.brick8_exact(),
    lambda: (W.brick_circuit(8, 4, 3, seed=0, cphase_between=False), W.sector_bitstrings_all(8, 4)),
    lambda: (W.random_fig4_circuit(8, 3, 5, 2, seed=21), W.sector_bitstrings_all(8, 3)),
    lambda: (W.random_fig4_circuit(10, 5, 6, 3, seed=22), W.sector_bitstrings_all(10, 5)),
    lambda: (W.random_fig4_circuit(7, 2, 4, 2, seed=23, angle_std=3.0), W.sector_bitstrings_all(7, 2)),
])
def test_exact_amplitudes_match_statevector(maker):
    c, bits = maker()
    amp = O.exact_amplitudes(c, bits)
    sv = O.statevector_amplitudes(c.n_modes, c.occupied_modes(), c.gates, _modes_list(bits))
    assert np.max(np.abs(amp - sv)) < 1e-12
    # the sector's probabilities sum to one (particle number is conserved)
    assert abs(np.sum(np.abs(amp) ** 2) - 1.0) < 1e-12


def test_exact_lucj_12_qubits_all_400_outcomes():
    """Fig. 7's shape: 6 orbitals, 3a+3b, one Jastrow layer with 12
    controlled-phase gates (6 on-site + 3 aa + 3 bb), angles N(pi, 0.1)."""
    c = W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1, math.pi), seed=7)
    assert c.n_cphase == 12
    bits = W.spin_sector_bitstrings_all(6, 3, 3)
    assert len(bits) == 400
    amp = O.exact_amplitudes(c, bits)
    sv = O.statevector_amplitudes(c.n_modes, c.occupied_modes(), c.gates, _modes_list(bits))
    assert np.max(np.abs(amp - sv)) < 1e-12
    # alpha and beta Hamming weights are conserved separately (Section VI-A):
    # the (3,3) sector alone already carries all the probability
    assert abs(np.sum(np.abs(amp) ** 2) - 1.0) < 1e-12


def test_two_layer_lucj_matches_statevector():
    c = W.lucj_circuit(5, 2, 2, 2, n_onsite=3, n_same=2, angle_sampler=W.normal_var(0.5), seed=8)
    bits = W.spin_sector_bitstrings_all(5, 2, 2)
    amp = O.exact_amplitudes(c, bits)
    sv = O.statevector_amplitudes(c.n_modes, c.occupied_modes(), c.gates, _modes_list(bits))
    assert np.max(np.abs(amp - sv)) < 1e-12


def test_wrong_weight_bitstring_has_zero_probability():
    c, _ = W.brick8_exact()
    bits = np.array([W.modes_to_bits([0, 1, 2]), W.modes_to_bits([0, 1, 2, 3, 4])], dtype=np.uint64)
    assert np.all(O.exact_probabilities(c, bits) == 0.0)


# --------------------------------------------------------------------------- closed forms


def test_k0_is_a_single_minor_of_the_network_unitary():
    """Terhal-DiVincenzo (Eq. 3): with no controlled-phase gate, <b|M|a> is the
    minor of the network's unitary, rows from b and columns from a. The unitary
    here is the generator's Haar draw, not a product the oracle formed."""
    rng = np.random.default_rng(5)
    V = W.haar_unitary(7, rng)
    c = W.Circuit(7, W.modes_to_bits([0, 2, 3]), W.make_gates(W.givens_network(V)))
    bits = W.sector_bitstrings_all(7, 3)
    amp = O.exact_amplitudes(c, bits)
    cols = [0, 2, 3]
    for b, a in zip(bits, amp):
        rows = W.bits_to_modes(b)
        assert abs(a - np.linalg.det(V[np.ix_(rows, cols)])) < 1e-12


def test_givens_network_reproduces_the_unitary():
    rng = np.random.default_rng(3)
    for n in (2, 5, 16):
        V = W.haar_unitary(n, rng)
        M = np.eye(n, dtype=np.complex128)
        for kind, p, q, theta, phi in W.givens_network(V):
            G = np.eye(n, dtype=np.complex128)
            if kind == W.PHASE:
                G[p, p] = np.exp(1j * phi)
            else:
                c, s = math.cos(theta), math.sin(theta)
                G[p, p], G[p, q], G[q, p], G[q, q] = c, -np.exp(1j * phi) * s, np.exp(-1j * phi) * s, c
            M = G @ M
        assert np.max(np.abs(M - V)) < 1e-12


def test_zero_angle_cphase_is_identity_and_angles_wrap():
    base, bits = W.brick8_exact()
    recs = [(int(g["kind"]), int(g["p"]), int(g["q"]), float(g["theta"]), float(g["phi"])) for g in base.gates]
    p0 = O.exact_probabilities(base, bits)
    with_zero = W.Circuit(8, base.occupation, W.make_gates(recs[:5] + [(W.CPHASE, 1, 6, 0.0, 0.0)] + recs[5:]))
    assert np.max(np.abs(O.exact_probabilities(with_zero, bits) - p0)) < 1e-14
    shifted = [(k, p, q, t + (4 * math.pi if k == W.CPHASE else 0.0), f) for (k, p, q, t, f) in recs]
    c2 = W.Circuit(8, base.occupation, W.make_gates(shifted))
    assert np.max(np.abs(O.exact_probabilities(c2, bits) - p0)) < 1e-13


def test_cphase_next_to_basis_states_does_not_change_probabilities():
    base, bits = W.brick8_exact()
    recs = [(int(g["kind"]), int(g["p"]), int(g["q"]), float(g["theta"]), float(g["phi"])) for g in base.gates]
    nocp = [r for r in recs if r[0] != W.CPHASE]
    p_ref = O.exact_probabilities(W.Circuit(8, base.occupation, W.make_gates(nocp)), bits)
    edge = [(W.CPHASE, 0, 5, 1.1, 0.0)] + nocp + [(W.CPHASE, 2, 7, -0.7, 0.0), (W.CPHASE, 3, 4, 2.9, 0.0)]
    p_edge = O.exact_probabilities(W.Circuit(8, base.occupation, W.make_gates(edge)), bits)
    assert np.max(np.abs(p_edge - p_ref)) < 1e-14


# --------------------------------------------------------------------------- extent, thresholds


def test_extent_all_pi_is_two_to_the_k():
    recs = [(W.CPHASE, 0, j + 1, math.pi, 0.0) for j in range(9)]
    assert abs(O.extent(W.make_gates(recs)) - 2.0 ** 9) < 1e-9


def test_printed_extents_reproduce_under_the_variance_reading():
    gold = _load("printed_extents.json")
    rng = np.random.default_rng(0)
    for case in gold["cases"]:
        k, mean, var = case["k"], case["mean"], case["var"]
        th = rng.normal(mean, math.sqrt(var), size=(20000, k))
        a = np.abs(np.vectorize(O.wrap_angle)(th)) / 4
        xi = np.prod((np.cos(a) + np.sin(a)) ** 2, axis=1)
        lo, hi = np.quantile(xi, [0.001, 0.999])
        assert lo <= case["printed"] <= hi, case["where"]
    # the standard-deviation reading of Fig. 5's N(0, 1e-3) cannot give 1.732
    th = rng.normal(0.0, 1e-3, size=(20000, 43))
    a = np.abs(th) / 4
    xi = np.prod((np.cos(a) + np.sin(a)) ** 2, axis=1)
    assert np.quantile(xi, 0.999) < 1.1


def test_fig3_worked_example():
    g = _load("fig3_trajectory_example.json")
    recs = [(W.CPHASE, 0, 1 + j, t, 0.0) for j, t in enumerate(g["theta"])]
    gates = W.make_gates(recs)
    cps = O.cphase_list(gates)
    assert [cp["pT1"] for cp in cps] == g["p_x1"]
    assert O.sampling_probability(gates, g["x"]) == g["P_x"]
    # the sampler draws x = 010 with frequency 1/4
    c = W.Circuit(4, W.modes_to_bits([0]), gates)
    X = O.sample_trajectories(c, b_index=0, t=40000, seed=12345)
    assert np.all(X[:, 0] == 0)
    f = np.mean(np.all(X == np.array(g["x"]), axis=1))
    assert abs(f - 0.25) < 4 * math.sqrt(0.25 * 0.75 / 40000)


def test_thresholds_match_eq_10_11():
    rng = np.random.default_rng(9)
    for theta in rng.uniform(-3 * math.pi, 3 * math.pi, size=50):
        cp = O.cphase_list(W.make_gates([(W.CPHASE, 0, 1, theta, 0.0)]))[0]
        a = abs(O.wrap_angle(theta)) / 4
        p1 = math.sin(a) / (math.sin(a) + math.cos(a))
        assert abs(cp["pT1"] - p1) <= 2.0 ** -32
        assert 0 < cp["T"] < 2 ** 31 + 1


def _eq6_decimal(eps, delta, pmax, xi):
    """Eq. 6 worked out in 40-digit decimal arithmetic (an independent
    evaluation: exact square roots and logarithm of the decimal inputs)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    E, D, P, X = (Decimal(repr(v)) for v in (eps, delta, pmax, xi))
    e2 = Decimal(1).exp() ** 2
    num = (X.sqrt() + P.sqrt()) ** 2
    den = ((P + E).sqrt() - P.sqrt()) ** 2
    v = 2 * num / den * (2 * e2 / D).ln()
    return int(v.to_integral_value(rounding="ROUND_CEILING")), v


@pytest.mark.parametrize("eps,delta,pmax,xi", [(0.01, 0.05, 0.0, 4.0), (0.02, 1e-3, 0.09, 2.25),
                                                (1e-4, 0.01, 3e-5, 6.7), (0.25, 0.5, 1.0, 1.0)])
def test_trajectory_bound_eq6_worked_values(eps, delta, pmax, xi):
    """Eq. 6 at four points against a 40-digit evaluation (values chosen away
    from integer boundaries)."""
    t_dec, v = _eq6_decimal(eps, delta, pmax, xi)
    assert abs(float(v) - round(float(v))) > 1e-6
    assert O.trajectory_count_bound(eps, delta, pmax, xi) == t_dec


def test_trajectory_bound_eq6_limits_and_monotonicity():
    """p_max = 0: 2 xi / eps log(2 e^2 / delta) (the denominator is eps);
    eps << p_max: ~ 8 p_max (sqrt xi + sqrt p_max)^2 / eps^2 log(2 e^2 / delta)
    ((sqrt(p + eps) - sqrt p)^2 -> eps^2 / (4 p)); monotone in every argument."""
    L = math.log(2 * math.e ** 2 / 1e-3)
    assert O.trajectory_count_bound(1e-2, 1e-3, 0.0, 4.0) == math.ceil(2 * 4.0 / 1e-2 * L)
    p, xi, eps = 0.3, 5.0, 1e-5
    approx = 8 * p * (math.sqrt(xi) + math.sqrt(p)) ** 2 / eps ** 2 * L
    assert abs(O.trajectory_count_bound(eps, 1e-3, p, xi) / approx - 1) < 1e-4
    base = (1e-3, 1e-2, 0.01, 3.0)
    t0 = O.trajectory_count_bound(*base)
    assert O.trajectory_count_bound(2e-3, 1e-2, 0.01, 3.0) < t0       # larger eps
    assert O.trajectory_count_bound(1e-3, 2e-2, 0.01, 3.0) < t0       # larger delta
    assert O.trajectory_count_bound(1e-3, 1e-2, 0.02, 3.0) > t0       # larger p_max
    assert O.trajectory_count_bound(1e-3, 1e-2, 0.01, 6.0) > t0       # larger extent


def test_splitmix64_known_answers():
    """The Estimate rounds' seeds come from SplitMix64; pinned to its published
    output sequence for state 0."""
    kat = json.load(open(os.path.join(GOLD, "splitmix64_kat.json")))
    g = 0x9E3779B97F4A7C15
    out = [O.splitmix64((k * g) & ((1 << 64) - 1)) for k in range(1, 5)]
    assert out == [int(h, 16) for h in kat["outputs_hex"]]


def test_trajectory_grid():
    """Counts round up to m * 2^e, 4 <= m <= 8: never down, at most 25 % up."""
    for t in list(range(1, 300)) + [1023, 1024, 1025, 10 ** 6 + 7, 2 ** 31 + 1]:
        g = O.trajectory_grid(t)
        assert g >= t and (t <= 8 or g <= 1.25 * t)
        e = max(0, g.bit_length() - 4)
        assert g % (1 << e) == 0 and (g >> e) <= 15


def test_estimate_oracle_meets_eps():
    """The oracle's Estimate on three bitstrings of the 8-mode brick circuit:
    within eps of the exact probability (failure probability 1e-3 each), with
    fewer trajectories than one Raw Estimate at p_max = 1 would take."""
    c, bits = W.brick8_exact()
    sub = bits[[3, 17, 40]]
    p = O.exact_probabilities(c, sub)
    eps, delta = 0.02, 1e-3
    ph, _, traj = O.estimate(c, sub, eps, delta, seed=11)
    assert np.all(np.abs(ph - p) <= eps)
    assert np.all(traj < O.trajectory_count_bound(eps, delta, 1.0, O.extent(c.gates)))


# --------------------------------------------------------------------------- Raw Estimate


def test_raw_estimate_zero_angles_is_exact():
    c, bits = W.brick8_exact()
    recs = [(int(g["kind"]), int(g["p"]), int(g["q"]), 0.0 if int(g["kind"]) == W.CPHASE else float(g["theta"]),
             float(g["phi"])) for g in c.gates]
    c0 = W.Circuit(8, c.occupation, W.make_gates(recs))
    p = O.exact_probabilities(c0, bits[:10])
    ph, se = O.raw_estimate(c0, bits[:10], t=17, seed=3)
    assert np.max(np.abs(ph - p)) < 1e-15
    assert np.all(se < 1e-12)


def test_raw_estimate_unbiased_amplitude_and_exact_bias_formula():
    """E[alpha_hat] = alpha and E[p_hat] = p + (E|Y|^2 - p)/t: z-tests over seeds."""
    c = W.random_fig4_circuit(6, 3, 5, 2, seed=31, angle_std=1.5)
    b = W.sector_bitstrings_all(6, 3)[7:8]
    alpha, m2 = O.expected_second_moment(c, b[0])
    p = abs(alpha) ** 2
    t, n_seeds = 32, 300
    ah = np.zeros(n_seeds, dtype=np.complex128)
    ph = np.zeros(n_seeds)
    for sd in range(n_seeds):
        p_hat, _, a_hat, _ = O.raw_estimate(c, b, t=t, seed=1000 + sd, return_details=True)
        ah[sd], ph[sd] = a_hat[0], p_hat[0]
    for comp, want in ((ah.real, alpha.real), (ah.imag, alpha.imag)):
        z = (comp.mean() - want) / (comp.std(ddof=1) / math.sqrt(n_seeds))
        assert abs(z) < 4.0
    z = (ph.mean() - (p + (m2 - p) / t)) / (ph.std(ddof=1) / math.sqrt(n_seeds))
    assert abs(z) < 4.0


def test_raw_estimate_converges_and_stderr_is_calibrated():
    c = W.random_fig4_circuit(6, 3, 5, 2, seed=32, angle_std=1.0)
    bits = W.sector_bitstrings_all(6, 3)[:6]
    p = O.exact_probabilities(c, bits)
    ph, se = O.raw_estimate(c, bits, t=20000, seed=77)
    z = (ph - p) / np.maximum(se, 1e-300)
    assert np.all(np.abs(z) < 5.0)


def test_raw_estimate_stderr_matches_spread_over_seeds():
    """The reported standard error is the standard deviation of p_hat over
    independent runs: over 300 seeds at t = 1024, the sample standard deviation
    of p_hat and the root mean square of the reported standard errors agree
    within 20 % for the four most probable outcomes (0.96-1.04 observed; the
    sampling error of the ratio is about 4 %)."""
    c = W.random_fig4_circuit(6, 3, 5, 2, seed=32, angle_std=1.5)
    bits = W.sector_bitstrings_all(6, 3)
    p = O.exact_probabilities(c, bits)
    for bi in np.argsort(-p)[:4]:
        runs = [O.raw_estimate(c, bits[bi:bi + 1], t=1024, seed=5000 + sd) for sd in range(300)]
        ph = np.array([r[0][0] for r in runs])
        se = np.array([r[1][0] for r in runs])
        ratio = ph.std(ddof=1) / math.sqrt(np.mean(se ** 2))
        assert 0.8 < ratio < 1.25, (int(bi), ratio)


def test_trajectories_depend_only_on_global_index():
    c, bits = W.brick8_exact()
    X1 = O.sample_trajectories(c, b_index=12345678901, t=64, seed=9)
    X2 = O.sample_trajectories(c, b_index=12345678901, t=64, seed=9)
    X3 = O.sample_trajectories(c, b_index=12345678902, t=64, seed=9)
    assert np.array_equal(X1, X2) and not np.array_equal(X1, X3)


# --------------------------------------------------------------------------- gradients


def test_forward_mode_gradient_matches_central_differences():
    c = W.random_fig4_circuit(6, 3, 4, 2, seed=41, angle_std=1.0)
    bits = W.sector_bitstrings_all(6, 3)[:8]
    rng = np.random.default_rng(4)
    g = rng.uniform(0, 1, len(bits))
    ang = O.get_angles(c.gates)
    grad = O.prob_gradient(c, bits, g)
    h = 1e-6
    fd = np.zeros(len(ang))
    for a in range(len(ang)):
        e = np.zeros(len(ang))
        e[a] = h
        cp = W.Circuit(c.n_modes, c.occupation, O.set_angles(c.gates, ang + e))
        cm = W.Circuit(c.n_modes, c.occupation, O.set_angles(c.gates, ang - e))
        fd[a] = np.dot(g, O.exact_probabilities(cp, bits) - O.exact_probabilities(cm, bits)) / (2 * h)
    assert np.max(np.abs(grad - fd)) <= 1e-7 * max(1.0, np.max(np.abs(grad)))


def test_forward_mode_derivative_of_amplitude_matches_statevector_differences():
    """The derivative of the full amplitude (with its global phase) against
    central differences of the brute-force state vector."""
    c = W.random_fig4_circuit(6, 2, 3, 2, seed=42, angle_std=1.0)
    bits = W.sector_bitstrings_all(6, 2)
    ang = O.get_angles(c.gates)
    rng = np.random.default_rng(1)
    v = rng.normal(size=len(ang))
    _, damp = O.exact_amplitudes(c, bits, with_global_phase=True, direction=v)
    h = 1e-6
    ap = O.statevector_amplitudes(6, c.occupied_modes(), O.set_angles(c.gates, ang + h * v), _modes_list(bits))
    am = O.statevector_amplitudes(6, c.occupied_modes(), O.set_angles(c.gates, ang - h * v), _modes_list(bits))
    assert np.max(np.abs(damp - (ap - am) / (2 * h))) < 1e-8
