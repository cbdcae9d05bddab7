"""Plain FP64 CPU oracle for ExtraFerm's Exact and Raw Estimate algorithms.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this module. It
shares no code with the CUDA library; the only module both sides use is
``workloads`` (seeded input generators, no method arithmetic).

What it computes (the paper's definitions, written out):

* Mode-transformation matrix (Section II-B, Eqs. 2-3). A passive gate acts on
  the single-particle space by an n x n matrix; a circuit's matrix is the
  product of its gates' matrices, each later gate multiplied on the left
  (column convention: column c holds the image of mode c). For basis states
  |a>, |b> of equal Hamming weight, <b|M|a> = det V[R, C] with rows R = set
  bits of b and columns C = set bits of a, both ascending.
* Controlled-phase decomposition (Section III-B, Eq. 7):
  c(theta) = e^{i theta/4} [cos(theta/4) d0(theta) + i sin(theta/4) d1(theta)].
  As a passive gate d_x(theta) = e^{-i theta/2} M(D_x) with the mode matrix
  D_x = diag((-1)^x e^{i theta/2} on modes p, q; 1 elsewhere), so a trajectory
  x replaces every controlled-phase gate by D_{x_j}, and the common scalar
  prod_j e^{-i theta_j/4} multiplies the amplitude.
* Exact (Eqs. 8-9): amp(b) = prod_j e^{-i theta_j/4} sum_x w(x) det U(x)[R, C],
  w(x) = prod_j cos(theta_j/4)^{1-x_j} (i sin(theta_j/4))^{x_j}
  (the printed exponent x_j - 1 is read as 1 - x_j: only that reproduces the
  state vector), p(b) = |amp(b)|^2.
* Branch matrices follow Section IV-B, Eq. 14, generalised to several runs of
  controlled-phase gates: U(x) = S_L D_L(x) ... S_1 D_1(x) S_0, where S_l is
  the ordered product of the passive gates between the (l)-th and (l+1)-th
  run and D_l(x) the (diagonal) product of the run's D_{x_j}.
* Extent (Eq. 5): xi = prod_j (cos(|theta_j|/4) + sin(|theta_j|/4))^2.
* Raw Estimate (Eqs. 10-12, Section III-A): per bitstring, t trajectories are
  drawn from P(x) = prod_j p(x_j), p(x_j = 1) = sin(|t_j|/4) /
  (sin(|t_j|/4) + cos(|t_j|/4)), by inverse-transform sampling with one
  uniform per gate; the estimate is p_hat = |alpha_hat|^2 with
  alpha_hat = (1/t) sum_s w(x_s)/P(x_s) det U(x_s)[R, C].

Readings where the paper is silent:

* Angles are wrapped to theta' in (-pi, pi] before the decomposition
  (c(theta) is 2 pi-periodic, the decomposition is not).
* Uniforms are 32-bit words of Philox4x32-10 (``oracle.philox``), word
  (j mod 4) of the block with counter (floor(j/4), s, b_lo, b_hi) and key
  (seed_lo, seed_hi); x_j = 1 iff u_j < T_j with the integer threshold
  T_j = round(p(x_j = 1) * 2^32), clamped to >= 1 when sin(theta'_j/4) != 0
  and 0 when it is 0. The importance weight uses the quantised
  p_T(1) = T_j / 2^32, p_T(0) = 1 - p_T(1), which keeps E[alpha_hat] exact.
* The Raw Estimate's standard error is the delta-method
  2 sqrt(Var_s[Re(conj(alpha_hat) Y_s)] / t) with the unbiased sample variance.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import trajectory_uniforms

GIVENS, PHASE, CPHASE = 0, 1, 2
TWO32 = 4294967296.0

# ---------------------------------------------------------------------------
# Angles and per-gate tables
# ---------------------------------------------------------------------------


def wrap_angle(theta: float) -> float:
    """theta' = theta - 2 pi m in (-pi, pi]."""
    t = theta - 2.0 * math.pi * math.floor((theta + math.pi) / (2.0 * math.pi))
    if t <= -math.pi:
        t += 2.0 * math.pi
    return t


def cphase_list(gates) -> list[dict]:
    """The controlled-phase gates in circuit order with their Eq. 7 / Eq. 10-12
    quantities (c = cos(theta'/4), s = sin(theta'/4), threshold T)."""
    out = []
    for gi, g in enumerate(gates):
        if int(g["kind"]) != CPHASE:
            continue
        th = wrap_angle(float(g["theta"]))
        c, s = math.cos(th / 4.0), math.sin(th / 4.0)
        sa, ca = math.sin(abs(th) / 4.0), math.cos(abs(th) / 4.0)
        p1 = sa / (sa + ca)
        if sa == 0.0:
            T = 0
        else:
            T = int(math.floor(p1 * TWO32 + 0.5))
            T = min(max(T, 1), 4294967295)
        pT1 = T / TWO32
        out.append(dict(gate=gi, p=int(g["p"]), q=int(g["q"]), theta=th, c=c, s=s,
                        p1=p1, T=T, pT1=pT1, pT0=1.0 - pT1))
    return out


def extent(gates) -> float:
    """Eq. 5."""
    xi = 1.0
    for cp in cphase_list(gates):
        a = abs(cp["theta"]) / 4.0
        xi *= (math.cos(a) + math.sin(a)) ** 2
    return xi


def trajectory_count_bound(eps: float, delta: float, p_max: float, xi: float) -> int:
    """Eq. 6: trajectories sufficient for |p_hat - p| <= eps with failure
    probability delta (the printed '= 1 - delta' read as '<= delta')."""
    num = (math.sqrt(xi) + math.sqrt(p_max)) ** 2
    den = (math.sqrt(p_max + eps) - math.sqrt(p_max)) ** 2
    return int(math.ceil(2.0 * num / den * math.log(2.0 * (math.e * math.e) / delta)))


def trajectory_grid(t: int) -> int:
    """Round a trajectory count up to m * 2^e with 4 <= m <= 8 (the Estimate
    driver's rounding, so that bitstrings with equal counts can share work)."""
    t = int(t)
    if t <= 8:
        return max(t, 1)
    e = t.bit_length() - 3
    m = -(-t // (1 << e))
    return m << e


def splitmix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014)."""
    mask = (1 << 64) - 1
    z &= mask
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return z ^ (z >> 31)


def estimate(circuit, bitstrings, eps: float, delta: float, seed: int, b_indices=None):
    """Estimate (Section III-A): |p_hat - p| <= eps with failure probability at
    most delta per bitstring, without a given p_max, by rounds of Raw Estimate
    that start loose and tighten. The paper describes the algorithm only in
    words (start from loose error and probability upper bounds, then call Raw
    Estimate iteratively); the schedule read here:

    * eps_0 = max(eps, 1/4), eps_r = max(eps, eps_0 / 2^r), rounds r = 0..R-1
      with R the first round at eps_r = eps; failure budget delta / R per round
      (union bound over the rounds);
    * round r gives each bitstring the Eq. 6 count for its own p_max (1 at
      first, then min(p_max, p_hat + eps_r) of the previous round), rounded up
      by ``trajectory_grid``, fresh trajectories from seed
      splitmix64(seed + (r + 1) * 0x9E3779B97F4A7C15), and the bitstring's
      global index;
    * the estimate is the last round's p_hat.

    Returns (p_hat, stderr, trajectories spent per bitstring)."""
    nb = len(bitstrings)
    if b_indices is None:
        b_indices = list(range(nb))
    xi = extent(circuit.gates)
    eps0 = max(eps, 0.25)
    R = 1
    while R < 64 and max(eps, eps0 / 2 ** (R - 1)) > eps:
        R += 1
    d_r = delta / R
    pmax = np.ones(nb)
    ph = np.zeros(nb)
    se = np.zeros(nb)
    traj = np.zeros(nb, dtype=np.int64)
    for r in range(R):
        eps_r = max(eps, eps0 / 2 ** r)
        seed_r = splitmix64(seed + (r + 1) * 0x9E3779B97F4A7C15)
        for i in range(nb):
            t = trajectory_grid(trajectory_count_bound(eps_r, d_r, float(pmax[i]), xi))
            p_i, se_i = raw_estimate(circuit, bitstrings[i:i + 1], t=t, seed=seed_r, b_indices=[b_indices[i]])
            ph[i], se[i] = p_i[0], se_i[0]
            pmax[i] = min(pmax[i], ph[i] + eps_r)
            traj[i] += t
    return ph, se, traj


def sampling_probability(gates, x_bits) -> float:
    """P_T(x) = prod_j p_T(x_j) with the quantised thresholds."""
    p = 1.0
    for cp, xj in zip(cphase_list(gates), x_bits):
        p *= cp["pT1"] if xj else cp["pT0"]
    return p


# ---------------------------------------------------------------------------
# Gate mode matrices and circuit structure
# ---------------------------------------------------------------------------


def givens_matrix(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -np.exp(1j * phi) * s], [np.exp(-1j * phi) * s, c]], dtype=np.complex128)


def givens_matrix_derivs(theta: float, phi: float):
    c, s = math.cos(theta), math.sin(theta)
    e, em = np.exp(1j * phi), np.exp(-1j * phi)
    d_theta = np.array([[-s, -e * c], [em * c, -s]], dtype=np.complex128)
    d_phi = np.array([[0.0, -1j * e * s], [-1j * em * s, 0.0]], dtype=np.complex128)
    return d_theta, d_phi


def angle_layout(gates) -> list[tuple[int, str]]:
    """Order of the differentiable angles: per gate in circuit order,
    Givens -> (theta, phi), PHASE -> phi, CPHASE -> theta."""
    out = []
    for gi, g in enumerate(gates):
        k = int(g["kind"])
        if k == GIVENS:
            out += [(gi, "theta"), (gi, "phi")]
        elif k == PHASE:
            out.append((gi, "phi"))
        else:
            out.append((gi, "theta"))
    return out


def get_angles(gates) -> np.ndarray:
    return np.array([float(gates[gi][name]) for gi, name in angle_layout(gates)])


def set_angles(gates, angles) -> np.ndarray:
    g2 = gates.copy()
    for (gi, name), a in zip(angle_layout(gates), angles):
        g2[gi][name] = a
    return g2


def segments_and_layers(n: int, gates, direction=None):
    """Split the circuit into passive segments S_0..S_L (each the ordered
    product of its gates' mode matrices) and diagonal layers (runs of
    consecutive controlled-phase gates, listed by their index among the
    controlled-phase gates). With ``direction`` (one value per angle of
    ``angle_layout``) also returns dS_l, the derivative of every S_l along it."""
    seg = np.eye(n, dtype=np.complex128)
    dseg = np.zeros((n, n), dtype=np.complex128)
    segs, dsegs, layers = [], [], []
    cur_layer = None
    ai = 0
    j = 0
    for g in gates:
        kind, p, q = int(g["kind"]), int(g["p"]), int(g["q"])
        if kind == CPHASE:
            if cur_layer is None:
                segs.append(seg)
                dsegs.append(dseg)
                cur_layer = []
            cur_layer.append(j)
            j += 1
            ai += 1
            continue
        if cur_layer is not None:
            layers.append(cur_layer)
            cur_layer = None
            seg = np.eye(n, dtype=np.complex128)
            dseg = np.zeros((n, n), dtype=np.complex128)
        G = np.eye(n, dtype=np.complex128)
        dG = np.zeros((n, n), dtype=np.complex128)
        if kind == GIVENS:
            if q != p + 1:
                raise ValueError("Givens rotations act on adjacent modes")
            th, ph = float(g["theta"]), float(g["phi"])
            G[np.ix_([p, q], [p, q])] = givens_matrix(th, ph)
            if direction is not None:
                dth, dph = givens_matrix_derivs(th, ph)
                dG[np.ix_([p, q], [p, q])] = direction[ai] * dth + direction[ai + 1] * dph
            ai += 2
        elif kind == PHASE:
            ph = float(g["phi"])
            G[p, p] = np.exp(1j * ph)
            if direction is not None:
                dG[p, p] = direction[ai] * 1j * np.exp(1j * ph)
            ai += 1
        else:
            raise ValueError(f"unknown gate kind {kind}")
        if direction is not None:
            dseg = dG @ seg + G @ dseg
        seg = G @ seg
    if cur_layer is not None:
        layers.append(cur_layer)
        seg = np.eye(n, dtype=np.complex128)
        dseg = np.zeros((n, n), dtype=np.complex128)
    segs.append(seg)
    dsegs.append(dseg)
    return segs, dsegs, layers


def _cphase_angle_slots(gates) -> list[int]:
    """Position of each controlled-phase gate's theta in ``angle_layout``."""
    slots = []
    for ai, (gi, _name) in enumerate(angle_layout(gates)):
        if int(gates[gi]["kind"]) == CPHASE:
            slots.append(ai)
    return slots


# ---------------------------------------------------------------------------
# Branch sums
# ---------------------------------------------------------------------------


def _det_derivative(A: np.ndarray, dA: np.ndarray) -> np.ndarray:
    """d det(A) along dA for a stack of square matrices, by multilinearity in
    the columns: sum_i det(A with column i replaced by dA's column i)."""
    eta = A.shape[-1]
    out = np.zeros(A.shape[:-2], dtype=np.complex128)
    for i in range(eta):
        Ai = A.copy()
        Ai[..., :, i] = dA[..., :, i]
        out += np.linalg.det(Ai)
    return out


class _Prepared:
    """Per-circuit quantities the oracle reuses across bitstrings."""

    def __init__(self, circuit, direction=None):
        self.n = int(circuit.n_modes)
        self.gates = circuit.gates
        self.cols = _bits_to_list(circuit.occupation)
        self.eta = len(self.cols)
        self.cps = cphase_list(self.gates)
        self.k = len(self.cps)
        self.segs, self.dsegs, self.layers = segments_and_layers(self.n, self.gates, direction)
        self.direction = direction
        self.cp_slots = _cphase_angle_slots(self.gates)
        self.global_phase = np.exp(-1j * sum(cp["theta"] for cp in self.cps) / 4.0)

    def branch_columns(self, X: np.ndarray):
        """U(x)[:, C] for a batch of trajectories (X: (B, k) of 0/1), and its
        derivative along ``direction`` if one was given."""
        B = X.shape[0]
        cols = self.cols
        Xm = np.broadcast_to(self.segs[0][:, cols], (B, self.n, self.eta)).copy()
        dXm = None
        if self.direction is not None:
            dXm = np.broadcast_to(self.dsegs[0][:, cols], (B, self.n, self.eta)).copy()
        for li, layer in enumerate(self.layers):
            d = np.ones((B, self.n), dtype=np.complex128)
            dd_coef = np.zeros((B, self.n), dtype=np.complex128)
            for j in layer:
                cp = self.cps[j]
                f = np.where(X[:, j] == 1, -1.0, 1.0) * np.exp(0.5j * cp["theta"])
                d[:, cp["p"]] *= f
                d[:, cp["q"]] *= f
                if self.direction is not None:
                    v = self.direction[self.cp_slots[j]]
                    dd_coef[:, cp["p"]] += 0.5j * v
                    dd_coef[:, cp["q"]] += 0.5j * v
            S, dS = self.segs[li + 1], self.dsegs[li + 1]
            Y = d[:, :, None] * Xm
            if self.direction is not None:
                dY = (d * dd_coef)[:, :, None] * Xm + d[:, :, None] * dXm
                dXm = dS @ Y + S @ dY
            Xm = S @ Y
        return Xm, dXm

    def weights(self, X: np.ndarray):
        """w(x) (Eq. 9, exponent read as 1 - x_j) and its derivative."""
        B = X.shape[0]
        w = np.ones(B, dtype=np.complex128)
        dw = np.zeros(B, dtype=np.complex128)
        for j, cp in enumerate(self.cps):
            one = X[:, j] == 1
            wj = np.where(one, 1j * cp["s"], cp["c"])
            if self.direction is not None:
                v = self.direction[self.cp_slots[j]]
                dwj = v * np.where(one, 1j * cp["c"] / 4.0, -cp["s"] / 4.0)
                dw = dw * wj + w * dwj
            w = w * wj
        return w, dw


def _bits_to_list(bits) -> list[int]:
    out = []
    for word in range(2):
        v = int(bits[word])
        while v:
            low = v & -v
            out.append(word * 64 + low.bit_length() - 1)
            v ^= low
    return out


def _all_branches(k: int, start: int, stop: int) -> np.ndarray:
    x = np.arange(start, stop, dtype=np.int64)
    return ((x[:, None] >> np.arange(k, dtype=np.int64)[None, :]) & 1).astype(np.int8)


def _chunk_size(prep: _Prepared, budget_bytes: float = 48e6) -> int:
    per = prep.n * prep.eta * 16 * (3 if prep.direction is not None else 1)
    return max(1, int(budget_bytes // per))


def exact_amplitudes(circuit, bitstrings, with_global_phase: bool = True, direction=None):
    """Exact algorithm (Eqs. 8-9). Returns amp(b) for every bitstring (rows of
    a (nb, 2) uint64 array) and, with ``direction``, d amp(b) along it.
    Bitstrings whose Hamming weight differs from the initial state's get 0."""
    prep = _Prepared(circuit, direction)
    nb = len(bitstrings)
    rows = [_bits_to_list(b) for b in bitstrings]
    amp = np.zeros(nb, dtype=np.complex128)
    damp = np.zeros(nb, dtype=np.complex128)
    valid = [i for i, r in enumerate(rows) if len(r) == prep.eta]
    if any(m >= prep.n for r in rows for m in r):
        raise ValueError("bitstring has a bit at or above n_modes")
    total = 1 << prep.k
    step = _chunk_size(prep)
    for start in range(0, total, step):
        X = _all_branches(prep.k, start, min(total, start + step))
        Xm, dXm = prep.branch_columns(X)
        w, dw = prep.weights(X)
        for i in valid:
            A = Xm[:, rows[i], :]
            dets = np.linalg.det(A)
            amp[i] += np.sum(w * dets)
            if direction is not None:
                ddet = _det_derivative(A, dXm[:, rows[i], :])
                damp[i] += np.sum(dw * dets + w * ddet)
    if with_global_phase:
        amp = amp * prep.global_phase
        if direction is not None:
            slots = prep.cp_slots
            dphase = -0.25j * sum(direction[s] for s in slots)
            damp = damp * prep.global_phase + amp * dphase
    if direction is not None:
        return amp, damp
    return amp


def exact_probabilities(circuit, bitstrings) -> np.ndarray:
    return np.abs(exact_amplitudes(circuit, bitstrings, with_global_phase=False)) ** 2


def prob_directional_derivative(circuit, bitstrings, grad_p, direction) -> float:
    """sum_b grad_p[b] * dp_b along ``direction`` (forward mode through the
    products, the determinants and the weights)."""
    amp, damp = exact_amplitudes(circuit, bitstrings, with_global_phase=False,
                                 direction=np.asarray(direction, dtype=np.float64))
    dp = 2.0 * np.real(np.conj(amp) * damp)
    return float(np.dot(np.asarray(grad_p, dtype=np.float64), dp))


def prob_gradient(circuit, bitstrings, grad_p, angle_indices=None) -> np.ndarray:
    """Gradient of L = sum_b grad_p[b] p_b with respect to the angles of
    ``angle_layout`` (or the subset ``angle_indices``), one forward-mode pass
    per angle. Slow: for small circuits and sampled components."""
    na = len(angle_layout(circuit.gates))
    idx = list(range(na)) if angle_indices is None else list(angle_indices)
    out = np.zeros(len(idx))
    for o, a in enumerate(idx):
        e = np.zeros(na)
        e[a] = 1.0
        out[o] = prob_directional_derivative(circuit, bitstrings, grad_p, e)
    return out


# ---------------------------------------------------------------------------
# Raw Estimate
# ---------------------------------------------------------------------------


def sample_trajectories(circuit, b_index: int, t: int, seed: int, s_start: int = 0) -> np.ndarray:
    """Trajectory bits x_s (shape (t, k), int8) of bitstring number ``b_index``
    by inverse-transform sampling (Eq. 12) with the quantised thresholds."""
    cps = cphase_list(circuit.gates)
    k = len(cps)
    if k == 0:
        return np.zeros((t, 0), dtype=np.int8)
    s = np.arange(s_start, s_start + t, dtype=np.uint64)
    u = trajectory_uniforms(seed, b_index, s, k)
    T = np.array([cp["T"] for cp in cps], dtype=np.uint64)[None, :]
    return (u < T).astype(np.int8)


def raw_estimate(circuit, bitstrings, t: int, seed: int, b_indices=None, return_details: bool = False,
                 return_scale: bool = False):
    """Raw Estimate for each bitstring; ``b_indices`` are the global bitstring
    indices that key the generator (default 0..nb-1). Returns (p_hat, stderr)
    or, with ``return_details``, also alpha_hat and the total flip count; with
    ``return_scale`` one more array, the mean |Y_i| over the trajectories (the
    magnitude against which rounding in the terms of the Eq. 11 average is
    measured)."""
    prep = _Prepared(circuit)
    nb = len(bitstrings)
    if b_indices is None:
        b_indices = list(range(nb))
    rows = [_bits_to_list(b) for b in bitstrings]
    ratio0 = np.array([cp["c"] / cp["pT0"] for cp in prep.cps])
    ratio1 = np.array([(cp["s"] / cp["pT1"]) if cp["T"] > 0 else 0.0 for cp in prep.cps])
    p_hat = np.zeros(nb)
    stderr = np.zeros(nb)
    alpha = np.zeros(nb, dtype=np.complex128)
    scale = np.zeros(nb)
    flips = 0
    step = _chunk_size(prep)
    for i in range(nb):
        if len(rows[i]) != prep.eta:
            continue
        Ys = []
        for s0 in range(0, t, step):
            tt = min(step, t - s0)
            X = sample_trajectories(circuit, int(b_indices[i]), tt, seed, s0)
            flips += int(X.sum())
            Xm, _ = prep.branch_columns(X)
            dets = np.linalg.det(Xm[:, rows[i], :])
            r = np.ones(tt, dtype=np.complex128)
            for j in range(prep.k):
                r = r * np.where(X[:, j] == 1, 1j * ratio1[j], ratio0[j])
            Ys.append(r * dets)
        Y = np.concatenate(Ys) if Ys else np.zeros(0, dtype=np.complex128)
        a = Y.mean()
        alpha[i] = a
        scale[i] = float(np.abs(Y).mean()) if len(Y) else 0.0
        p_hat[i] = abs(a) ** 2
        if t > 1:
            z = np.real(np.conj(a) * Y)
            stderr[i] = 2.0 * math.sqrt(max(z.var(ddof=1), 0.0) / t)
    extra = (scale,) if return_scale else ()
    if return_details:
        return (p_hat, stderr, alpha, flips) + extra
    return (p_hat, stderr) + extra


def expected_second_moment(circuit, bitstring) -> tuple[complex, float]:
    """For small k: alpha = sum_x w(x) det and E_P|Y|^2 = sum_x |w(x)|^2 |det|^2 / P_T(x),
    by enumeration (used to test the Raw Estimate's exact bias formula)."""
    prep = _Prepared(circuit)
    rows = _bits_to_list(bitstring)
    X = _all_branches(prep.k, 0, 1 << prep.k)
    Xm, _ = prep.branch_columns(X)
    dets = np.linalg.det(Xm[:, rows, :])
    w, _ = prep.weights(X)
    P = np.ones(len(X))
    for j, cp in enumerate(prep.cps):
        P = P * np.where(X[:, j] == 1, cp["pT1"], cp["pT0"])
    alpha = np.sum(w * dets)
    keep = P > 0
    m2 = float(np.sum(np.abs(w[keep] * dets[keep]) ** 2 / P[keep]))
    return complex(alpha), m2
