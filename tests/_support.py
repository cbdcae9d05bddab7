"""Helpers shared by the GPU parity tests (no fixtures)."""
import math

import numpy as np

import oracle as O
import workloads as W


def likely_bitstrings(c, nb, seed, pool=400):
    """nb bitstrings that carry probability: the most probable (by the oracle)
    of a pool of one- to three-particle moves, each by at most 4 modes, away
    from the initial occupation."""
    rng = np.random.default_rng(seed)
    occ0 = c.occupied_modes()
    cand = set()
    for _ in range(20 * pool):
        if len(cand) >= pool:
            break
        occ = set(occ0)
        for _ in range(int(rng.integers(1, 4))):
            m = int(rng.choice(sorted(occ)))
            t = m + int(rng.integers(-4, 5))
            if 0 <= t < c.n_modes and t not in occ:
                occ.remove(m)
                occ.add(t)
        cand.add(tuple(sorted(occ)))
    bits = np.array([W.modes_to_bits(m) for m in sorted(cand)], dtype=np.uint64)
    p = O.exact_probabilities(c, bits)
    return bits[np.argsort(-p)[:nb]]


def neutral_gates_circuit():
    """8 modes, modes 0-3 occupied: two controlled-phase gates before any
    rotation, one on modes 3, 4 after two brick layers (with a third to
    follow), one after the last rotation. Returns the circuit and the angle
    slots of the first, second and fourth gate (probability-neutral) and of
    the third."""
    rng = np.random.default_rng(31)
    recs = [(W.CPHASE, 0, 5, 0.7, 0.0), (W.CPHASE, 3, 4, -0.9, 0.0)]
    def bricks():
        for start in (0, 1):
            for p in range(start, 7, 2):
                recs.append((W.GIVENS, p, p + 1, *rng.uniform(0, 2 * math.pi, 2)))
    bricks()
    bricks()
    recs.append((W.CPHASE, 3, 4, 1.1, 0.0))
    bricks()
    recs.append((W.CPHASE, 1, 6, 0.5, 0.0))
    c = W.Circuit(8, W.modes_to_bits([0, 1, 2, 3]), W.make_gates(recs))
    lay = O.angle_layout(c.gates)
    cp = [s for s, (gi, _) in enumerate(lay) if int(c.gates[gi]["kind"]) == W.CPHASE]
    return c, [cp[0], cp[1], cp[3]], cp[2]


def mixed_settled_circuit():
    """8 modes, modes 0-3 occupied. A controlled phase on modes 0 and 7 sits
    after every rotation that touches mode 7 and before every rotation that
    touches mode 0: mode 0 is settled before the gate and mode 7 after it, so
    the gate changes no probability. A second controlled phase (on modes 3, 4,
    between rotations of both) does. Returns the circuit and the angle slots
    of the two gates (neutral, active)."""
    rng = np.random.default_rng(41)
    recs = []
    for start in (1, 2, 1, 2):  # rotations on modes 1..7, none on mode 0
        for p in range(start, 7, 2):
            recs.append((W.GIVENS, p, p + 1, *rng.uniform(0, 2 * math.pi, 2)))
    recs.append((W.CPHASE, 0, 7, 1.3, 0.0))
    recs.append((W.CPHASE, 3, 4, -0.8, 0.0))
    for start in (0, 1, 0):  # rotations on modes 0..6, none on mode 7
        for p in range(start, 6, 2):
            recs.append((W.GIVENS, p, p + 1, *rng.uniform(0, 2 * math.pi, 2)))
    c = W.Circuit(8, W.modes_to_bits([0, 1, 2, 3]), W.make_gates(recs))
    lay = O.angle_layout(c.gates)
    cp = [s for s, (gi, _) in enumerate(lay) if int(c.gates[gi]["kind"]) == W.CPHASE]
    return c, cp[0], cp[1]
