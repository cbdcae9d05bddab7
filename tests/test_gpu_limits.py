"""GPU parity at the size limits of the interface and of each kernel path,
against the FP64 CPU oracle:

  * 128 modes, the largest circuit the two-word bitstrings address, with
    occupied modes on both words;
  * particle counts past the thread-per-minor LUs (eta = 12 and 20 per block:
    the warp-row LU with 16 and 32 lanes per minor);
  * the largest Raw Estimate block with FP32 minors (eta = 13) and with FP64
    minors (eta = 8).

Tolerances as in the other parity tests: 1e-10 (FP64) and 1e-5 (EF_PREC_AUTO)
relative to max(p, p_floor); the FP32-minor Raw Estimate alone (blocks of 13
particles have no FP64 recompute) relative to the squared mean |Y_s| of its
terms, with its error estimate bounding the observed error."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from _support import likely_bitstrings

pytestmark = pytest.mark.gpu


def _floor(c):
    return 1e-6 / math.comb(c.n_modes, len(c.occupied_modes()))


def _exact(lib, c, bits, prec):
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=prec)
    try:
        return lib.ef_prob_exact(h, bits)
    finally:
        lib.ef_circuit_destroy(h)


def _shifted(c, n_modes, offset):
    """c moved onto modes offset .. offset + c.n_modes - 1 of an n_modes circuit."""
    g = c.gates.copy()
    g["p"] += offset
    g["q"] += offset
    return W.Circuit(n_modes, W.modes_to_bits([m + offset for m in c.occupied_modes()]), g)


def _n128():
    # a 16-mode circuit placed on modes 56..71, across the two bitstring words
    c = _shifted(W.random_fig4_circuit(16, 4, 4, 3, seed=41), 128, 56)
    return c, likely_bitstrings(c, 24, 5)


def _big_eta(n, eta, k, seed, nb):
    c = W.random_fig4_circuit(n, eta, k, 2, seed=seed)
    return c, likely_bitstrings(c, nb, 5)


CASES = [
    ("n128-eta4-k4", _n128),
    ("n24-eta12-k4", lambda: _big_eta(24, 12, 4, 42, 24)),
    ("n40-eta20-k3", lambda: _big_eta(40, 20, 3, 43, 12)),
]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_exact_at_size_limits(lib, name, maker):
    c, bits = maker()
    if c.n_modes > 64:  # both words of the bitstrings are used
        assert np.any(bits[:, 1] != 0) and np.any(bits[:, 0] != 0)
    p_ref = O.exact_probabilities(c, bits)
    assert np.count_nonzero(p_ref > 1e-12) >= len(bits) // 2  # the bitstrings carry probability
    floor = _floor(c)
    for prec, tol in ((lib.EF_PREC_FP64, 1e-10), (lib.EF_PREC_AUTO, 1e-5)):
        p = _exact(lib, c, bits, prec)
        assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, floor)) <= tol, (name, prec)


@pytest.mark.parametrize("eta,prec", [(13, "fp32"), (8, "fp64"), (8, "auto")])
def test_approx_largest_blocks(lib, eta, prec):
    n = 2 * eta
    c = W.random_fig4_circuit(n, eta, 5, 2, seed=44 + eta, angle_std=1.0)
    bits = W.sector_bitstrings(n, eta, 6, np.random.default_rng(6))
    t, seed = 300, 0xABC
    p_ref, _, _, _, scale = O.raw_estimate(c, bits, t=t, seed=seed, return_details=True, return_scale=True)
    precision = {"fp64": lib.EF_PREC_FP64, "fp32": lib.EF_PREC_FP32_MINOR, "auto": lib.EF_PREC_AUTO}[prec]
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=precision)
    try:
        p, _, err = lib.ef_prob_approx(h, bits, t, seed=seed, want_err=True)
    finally:
        lib.ef_circuit_destroy(h)
    floor = _floor(c)
    rel = np.abs(p - p_ref) / np.maximum(p_ref, floor)
    if prec == "fp64":
        assert np.max(rel) <= 1e-10
    elif prec == "auto":
        assert np.max(rel) <= 1e-5
    else:
        assert np.max(np.abs(p - p_ref) / np.maximum(scale * scale, floor)) <= 1e-5
        assert np.all(rel <= err + 1e-9)
