"""Helpers shared by the GPU parity tests (no fixtures)."""
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
