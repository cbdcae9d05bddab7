"""Seeded synthetic inputs for the extended-matchgate probability path.

This module only *generates inputs*: gate lists (circuits of Givens rotations,
single-mode phases and controlled-phase gates), initial occupations and
bitstrings. It holds none of the method's arithmetic (no mode-transformation
matrices of trajectories, no minors, no branch sums, no sampling of
trajectories). Both the CPU oracle and the CUDA path consume what it returns.

Conventions shared by every consumer (they define the inputs, not the method):

* A gate is a record ``(kind, p, q, theta, phi)`` with ``kind`` one of
  ``GIVENS``, ``PHASE``, ``CPHASE``.
* ``GIVENS`` acts on adjacent modes ``q = p + 1`` with the 2x2 single-particle
  matrix ``[[cos t, -e^{i f} sin t], [e^{-i f} sin t, cos t]]`` (t = theta,
  f = phi) on rows/columns ``(p, q)``.
* ``PHASE`` multiplies mode ``p`` by ``e^{i phi}``.
* ``CPHASE`` is ``diag(1, 1, 1, e^{i theta})`` on the qubits of modes ``p != q``
  (Section III-B, Eq. 7).
* Bit ``m`` of a bitstring is the occupation of mode ``m``; bitstrings are two
  little-endian 64-bit words (modes 0-63, 64-127).
* LUCJ layouts put alpha spin-orbitals on modes ``0..norb-1`` and beta on
  ``norb..2*norb-1`` (Section VI-A writes the state as |beta alpha>).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GIVENS, PHASE, CPHASE = 0, 1, 2

GATE_DTYPE = np.dtype(
    [("kind", "<i4"), ("p", "<i4"), ("q", "<i4"), ("reserved", "<i4"),
     ("theta", "<f8"), ("phi", "<f8")]
)


@dataclass
class Circuit:
    """A particle-number-conserving extended matchgate circuit (an input)."""

    n_modes: int
    occupation: np.ndarray  # uint64[2], bit m = mode m occupied initially
    gates: np.ndarray  # GATE_DTYPE records, in circuit order
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_cphase(self) -> int:
        return int(np.count_nonzero(self.gates["kind"] == CPHASE))

    def occupied_modes(self) -> list[int]:
        return bits_to_modes(self.occupation)


def make_gates(records) -> np.ndarray:
    g = np.zeros(len(records), dtype=GATE_DTYPE)
    for i, (kind, p, q, theta, phi) in enumerate(records):
        g[i] = (kind, p, q, 0, theta, phi)
    return g


def modes_to_bits(modes) -> np.ndarray:
    w = np.zeros(2, dtype=np.uint64)
    for m in modes:
        w[m >> 6] |= np.uint64(1) << np.uint64(m & 63)
    return w


def bits_to_modes(bits) -> list[int]:
    out = []
    for word in range(2):
        v = int(bits[word])
        while v:
            low = v & -v
            out.append(word * 64 + low.bit_length() - 1)
            v ^= low
    return out


# ---------------------------------------------------------------------------
# Random orbital rotations as nearest-neighbour Givens networks
# ---------------------------------------------------------------------------

def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random n x n unitary (QR of a complex Ginibre matrix with the
    phases of R's diagonal divided out, Mezzadri 2007)."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def givens_network(V: np.ndarray, offset: int = 0) -> list[tuple]:
    """Gate records whose product (later gates multiplied on the left) is V.

    A triangular elimination with adjacent-row rotations reduces V to a
    diagonal of phases, column by column from the bottom up:
    n(n-1)/2 Givens rotations plus n single-mode phases. The returned circuit
    applies the phases first, then the inverse rotations in reverse order.
    """
    n = V.shape[0]
    W = np.array(V, dtype=np.complex128, copy=True)
    rots = []
    for c in range(n - 1):
        for i in range(n - 2, c - 1, -1):
            a, b = W[i, c], W[i + 1, c]
            if abs(b) == 0.0:
                theta, phi = 0.0, 0.0
            else:
                theta = math.atan2(abs(b), abs(a))
                phi = float(np.angle(-a * np.conj(b))) if abs(a) > 0 else 0.0
            ct, st = math.cos(theta), math.sin(theta)
            g = np.array([[ct, -np.exp(1j * phi) * st], [np.exp(-1j * phi) * st, ct]])
            W[[i, i + 1], :] = g @ W[[i, i + 1], :]
            rots.append((i, theta, phi))
    phases = np.angle(np.diag(W))
    recs = [(PHASE, offset + p, offset + p, 0.0, float(phases[p])) for p in range(n)]
    # g(theta, phi)^dagger = g(-theta, phi)
    recs += [(GIVENS, offset + i, offset + i + 1, -theta, phi) for (i, theta, phi) in reversed(rots)]
    return recs


def inverse_records(recs: list[tuple]) -> list[tuple]:
    """Records of the inverse of a Givens/phase network (reverse order, each gate inverted)."""
    out = []
    for kind, p, q, theta, phi in reversed(recs):
        if kind == GIVENS:
            out.append((GIVENS, p, q, -theta, phi))
        elif kind == PHASE:
            out.append((PHASE, p, q, 0.0, -phi))
        else:
            raise ValueError("only Givens/phase networks can be inverted here")
    return out


# ---------------------------------------------------------------------------
# Workload circuits
# ---------------------------------------------------------------------------

def brick_circuit(n_modes: int = 8, eta: int = 4, k: int = 3, seed: int = 0,
                  cphase_max: float = math.pi / 4, cphase_between: bool = True) -> Circuit:
    """One brick-wall layer of nearest-neighbour Givens rotations (angles
    theta, phi uniform in [0, 2 pi)) with k controlled-phase gates on random
    distinct mode pairs (angles uniform in [0, cphase_max]).

    With ``cphase_between`` the controlled-phase gates sit between the even
    and the odd bonds of the layer; otherwise they follow the whole layer.
    """
    rng = np.random.default_rng(seed)
    even = [(GIVENS, p, p + 1, *rng.uniform(0, 2 * math.pi, 2)) for p in range(0, n_modes - 1, 2)]
    odd = [(GIVENS, p, p + 1, *rng.uniform(0, 2 * math.pi, 2)) for p in range(1, n_modes - 1, 2)]
    cps = []
    for _ in range(k):
        p, q = rng.choice(n_modes, size=2, replace=False)
        cps.append((CPHASE, int(p), int(q), float(rng.uniform(0, cphase_max)), 0.0))
    recs = even + cps + odd if cphase_between else even + odd + cps
    return Circuit(n_modes, modes_to_bits(range(eta)), make_gates(recs),
                   name=f"brick-n{n_modes}-eta{eta}-k{k}")


def random_fig4_circuit(n_modes: int, eta: int, k: int, depth: int, seed: int,
                        angle_std: float = 1.0) -> Circuit:
    """Random particle-number-conserving extended matchgate circuit: ``depth``
    brick layers of Givens rotations with the k controlled-phase gates spread
    between layers on random (not necessarily adjacent) mode pairs."""
    rng = np.random.default_rng(seed)
    recs = []
    slots = sorted(rng.integers(0, depth + 1, size=k).tolist())
    si = 0
    for layer in range(depth + 1):
        while si < k and slots[si] == layer:
            p, q = rng.choice(n_modes, size=2, replace=False)
            recs.append((CPHASE, int(p), int(q), float(rng.normal(0.0, angle_std)), 0.0))
            si += 1
        if layer == depth:
            break
        for start in (0, 1):
            for p in range(start, n_modes - 1, 2):
                recs.append((GIVENS, p, p + 1, *rng.uniform(0, 2 * math.pi, 2)))
    return Circuit(n_modes, modes_to_bits(range(eta)), make_gates(recs),
                   name=f"random-n{n_modes}-eta{eta}-k{k}-d{depth}")


def jastrow_records(norb: int, n_onsite: int, n_same: int, angles: np.ndarray) -> list[tuple]:
    """Controlled-phase gates of one LUCJ Jastrow layer: ``n_same`` alpha-alpha
    pairs (p, p+1), ``n_same`` beta-beta pairs, and ``n_onsite`` opposite-spin
    on-site pairs (p, norb + p). ``angles`` has 2*n_same + n_onsite entries."""
    pairs = [(p, p + 1) for p in range(n_same)]
    pairs += [(norb + p, norb + p + 1) for p in range(n_same)]
    pairs += [(p, norb + p) for p in range(n_onsite)]
    assert len(angles) == len(pairs)
    return [(CPHASE, p, q, float(t), 0.0) for (p, q), t in zip(pairs, angles)]


def lucj_circuit(norb: int, n_alpha: int, n_beta: int, n_layers: int,
                 n_onsite: int, n_same: int, angle_sampler, seed: int,
                 inverse_final: bool = False, name: str = "") -> Circuit:
    """LUCJ-shaped circuit (Section IV-B, Eq. 13) on 2*norb modes.

    Orbital rotations are Haar-random norb x norb unitaries, one independent
    draw per spin and per rotation, each applied as a Givens network on its
    spin block. ``n_layers`` Jastrow layers of controlled-phase gates sit
    between the ``n_layers + 1`` rotations. With ``inverse_final`` and one
    layer the last rotation is the inverse of the first (rotation, Jastrow
    layer, inverse rotation).
    """
    rng = np.random.default_rng(seed)
    n = 2 * norb
    occ = modes_to_bits(list(range(n_alpha)) + [norb + p for p in range(n_beta)])
    rot_recs = []
    for r in range(n_layers + 1):
        if inverse_final and r == n_layers:
            rot_recs.append(inverse_records(rot_recs[0]))
            continue
        ua = haar_unitary(norb, rng)
        ub = haar_unitary(norb, rng)
        rot_recs.append(givens_network(ua, 0) + givens_network(ub, norb))
    recs = list(rot_recs[0])
    n_per_layer = 2 * n_same + n_onsite
    for layer in range(n_layers):
        recs += jastrow_records(norb, n_onsite, n_same, angle_sampler(rng, n_per_layer))
        recs += rot_recs[layer + 1]
    return Circuit(n, occ, make_gates(recs), name=name or f"lucj-{norb}o-{n_alpha}a{n_beta}b-L{n_layers}",
                   meta={"norb": norb, "n_alpha": n_alpha, "n_beta": n_beta})


def normal_var(var: float, mean: float = 0.0):
    """Sampler of N(mean, var): the second argument of N(., .) is a variance
    (the printed extents of Fig. 5, 7 and 8 reproduce only under that reading)."""
    std = math.sqrt(var)
    return lambda rng, m: rng.normal(mean, std, size=m)


def uniform_range(lo: float, hi: float):
    return lambda rng, m: rng.uniform(lo, hi, size=m)


# ---------------------------------------------------------------------------
# Bitstrings
# ---------------------------------------------------------------------------

def sector_bitstrings_all(n_modes: int, eta: int) -> np.ndarray:
    """Every bitstring of Hamming weight eta on n_modes modes (n_modes <= 64),
    in increasing integer order; shape (count, 2) uint64."""
    from itertools import combinations
    rows = [modes_to_bits(c) for c in combinations(range(n_modes), eta)]
    return np.array(rows, dtype=np.uint64).reshape(-1, 2)


def spin_sector_bitstrings_all(norb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    from itertools import combinations
    rows = []
    for cb in combinations(range(norb), n_beta):
        for ca in combinations(range(norb), n_alpha):
            rows.append(modes_to_bits(list(ca) + [norb + p for p in cb]))
    return np.array(rows, dtype=np.uint64).reshape(-1, 2)


def spin_sector_bitstrings(norb: int, n_alpha: int, n_beta: int, count: int,
                           rng: np.random.Generator) -> np.ndarray:
    """``count`` bitstrings uniform in the (n_alpha, n_beta) sector: independent
    uniform alpha and beta occupation subsets."""
    out = np.zeros((count, 2), dtype=np.uint64)
    for i in range(count):
        a = rng.choice(norb, size=n_alpha, replace=False)
        b = rng.choice(norb, size=n_beta, replace=False)
        out[i] = modes_to_bits([int(m) for m in a] + [norb + int(m) for m in b])
    return out


def sector_bitstrings(n_modes: int, eta: int, count: int, rng: np.random.Generator) -> np.ndarray:
    out = np.zeros((count, 2), dtype=np.uint64)
    for i in range(count):
        out[i] = modes_to_bits([int(m) for m in rng.choice(n_modes, size=eta, replace=False)])
    return out


# ---------------------------------------------------------------------------
# The five workload configurations
# ---------------------------------------------------------------------------

def brick8_exact() -> tuple[Circuit, np.ndarray]:
    """Exact mode, FP64: 8 modes, eta=4 in modes 0-3, one brick layer (seed 0),
    k=3 controlled-phase gates with angles in [0, pi/4]; all 70 bitstrings."""
    c = brick_circuit(8, 4, 3, seed=0)
    return c, sector_bitstrings_all(8, 4)


def lucj32_exact(n_bitstrings: int = 10_000) -> tuple[Circuit, np.ndarray]:
    """LUCJ-shaped exact mode: 2x16 modes, 8a+8b, one Jastrow layer of k=16
    (4 aa + 4 bb nearest-neighbour, 8 ab on-site) with angles N(0, 0.1)
    between a Haar rotation and its inverse; bitstrings uniform in (8,8)."""
    c = lucj_circuit(16, 8, 8, 1, n_onsite=8, n_same=4, angle_sampler=normal_var(0.1),
                     seed=2, inverse_final=True, name="lucj-32q-8a8b-k16")
    bits = spin_sector_bitstrings(16, 8, 8, n_bitstrings, np.random.default_rng(1002))
    return c, bits


def lucj52_approx(n_bitstrings: int = 100_000) -> tuple[Circuit, np.ndarray]:
    """Approximate mode: 2x26 modes, 5a+5b, 2-layer LUCJ with 26 on-site +
    25 aa + 25 bb controlled-phase gates per layer (k=152), angles uniform in
    [-0.05, 0.05]; bitstrings uniform in (5,5)."""
    c = lucj_circuit(26, 5, 5, 2, n_onsite=26, n_same=25, angle_sampler=uniform_range(-0.05, 0.05),
                     seed=3, name="lucj-52q-5a5b-k152")
    bits = spin_sector_bitstrings(26, 5, 5, n_bitstrings, np.random.default_rng(1003))
    return c, bits


def lucj52_trajectories(extent: float, eps: float = 1e-2, cap: int = 1_000_000) -> int:
    """t = ceil(extent * eps^-2), capped."""
    return int(min(math.ceil(extent / (eps * eps)), cap))


def lucj40_grad(n_bitstrings: int = 4096) -> tuple[Circuit, np.ndarray, np.ndarray]:
    """Differentiation: 2x20 modes, 6a+6b, 2-layer LUCJ with k=12 (per layer
    4 on-site + 1 aa + 1 bb), angles N(0, 0.1); 4096 sector bitstrings and
    weights uniform in [0, 1]."""
    c = lucj_circuit(20, 6, 6, 2, n_onsite=4, n_same=1, angle_sampler=normal_var(0.1),
                     seed=5, name="lucj-40q-6a6b-k12")
    rng = np.random.default_rng(1005)
    bits = spin_sector_bitstrings(20, 6, 6, n_bitstrings, rng)
    w = rng.uniform(0.0, 1.0, size=n_bitstrings)
    return c, bits, w


def uneven_batch64(n_circuits: int = 64, seed: int = 4) -> list[tuple[Circuit, np.ndarray, str]]:
    """Uneven batch: n uniform in even {12..40} (n/2 orbitals per spin), eta per
    spin uniform in [2, n/3], k uniform in [4, 24] with angles N(0, 0.1),
    1-3 Givens brick layers per spin, bitstrings per circuit log-uniform in
    [1e2, 1e5]; exact mode when k <= 14, approximate otherwise."""
    rng = np.random.default_rng(seed)
    out = []
    for ci in range(n_circuits):
        n = int(rng.choice(np.arange(12, 41, 2)))
        norb = n // 2
        eta = int(rng.integers(2, max(2, n // 3) + 1))
        eta = min(eta, norb)
        k = int(rng.integers(4, 25))
        depth = int(rng.integers(1, 4))
        recs = []
        # spin-separated brick layers with the controlled-phase gates between them
        cut = sorted(rng.integers(0, depth + 1, size=k).tolist())
        ki = 0
        for layer in range(depth + 1):
            while ki < k and cut[ki] == layer:
                if rng.uniform() < 0.5:
                    p = int(rng.integers(0, norb))
                    pair = (p, norb + p)
                else:
                    s = int(rng.integers(0, 2)) * norb
                    p = int(rng.integers(0, norb - 1))
                    pair = (s + p, s + p + 1)
                recs.append((CPHASE, pair[0], pair[1], float(rng.normal(0.0, math.sqrt(0.1))), 0.0))
                ki += 1
            if layer == depth:
                break
            for s in (0, norb):
                for start in (0, 1):
                    for p in range(start, norb - 1, 2):
                        recs.append((GIVENS, s + p, s + p + 1, *rng.uniform(0, 2 * math.pi, 2)))
        occ = modes_to_bits(list(range(eta)) + [norb + p for p in range(eta)])
        c = Circuit(n, occ, make_gates(recs), name=f"batch{ci}-n{n}-eta{eta}-k{k}-d{depth}")
        nb = int(round(10 ** rng.uniform(2.0, 5.0)))
        bits = spin_sector_bitstrings(norb, eta, eta, nb, rng)
        out.append((c, bits, "exact" if k <= 14 else "approx"))
    return out
