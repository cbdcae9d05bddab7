"""Planted mistakes in the oracle, on the CPU only: each mutant below is the
oracle's source with one plausible error (a dropped factor i, a wrong sign or
index, a transposed operand, a misread formula) and must make at least one of
the pins in test_oracle_pins.py fail. The pins therefore check the oracle
against the paper and the mathematics rather than against itself. Nothing here
touches the CUDA path."""
import inspect
import types

import pytest

import oracle
import oracle.extraferm_oracle as EO
import oracle.philox as PH
import test_oracle_pins as PINS

# (name, module, text in the oracle's source, replacement, pins expected to catch it)
MUTANTS = [
    ("weight without the factor i (Eq. 9)", EO,
     'wj = np.where(one, 1j * cp["s"], cp["c"])', 'wj = np.where(one, cp["s"], cp["c"])',
     ["exact_vs_statevector", "lucj12", "fd_gradient"]),
    ("exponent of cos read literally as x_j - 1 (Eq. 9)", EO,
     'wj = np.where(one, 1j * cp["s"], cp["c"])', 'wj = np.where(one, 1j * cp["s"], 1.0 / cp["c"])',
     ["exact_vs_statevector", "lucj12"]),
    ("phase e^{-i theta/2} instead of e^{+i theta/2} in D_x (Eq. 7)", EO,
     'np.exp(0.5j * cp["theta"])', 'np.exp(-0.5j * cp["theta"])',
     ["exact_vs_statevector", "lucj12"]),
    ("sign (-1)^x_j applied to one mode of the pair only (Eq. 7)", EO,
     'd[:, cp["q"]] *= f', 'd[:, cp["q"]] *= np.abs(f) * np.exp(0.5j * cp["theta"])',
     ["exact_vs_statevector", "lucj12"]),
    ("sin(|theta|/4) in the branch weight", EO,
     "c, s = math.cos(th / 4.0), math.sin(th / 4.0)", "c, s = math.cos(th / 4.0), math.sin(abs(th) / 4.0)",
     ["exact_vs_statevector", "lucj12"]),
    ("transposed first segment (rows and columns of Eq. 3 exchanged)", EO,
     "self.segs[0][:, cols]", "self.segs[0].T[:, cols]",
     ["exact_vs_statevector", "k0_minor"]),
    ("gates multiplied in the wrong order", EO,
     "seg = G @ seg", "seg = seg @ G",
     ["exact_vs_statevector", "k0_minor"]),
    ("Givens phase on the wrong off-diagonal element", EO,
     "[[c, -np.exp(1j * phi) * s], [np.exp(-1j * phi) * s, c]]",
     "[[c, -np.exp(-1j * phi) * s], [np.exp(1j * phi) * s, c]]",
     ["exact_vs_statevector", "k0_minor"]),
    ("angles wrapped into [0, 2 pi) instead of (-pi, pi]", EO,
     "math.floor((theta + math.pi) / (2.0 * math.pi))", "math.floor(theta / (2.0 * math.pi))",
     # Exact probabilities and the extent are unchanged by theta -> 2 pi - |theta| (c(theta) is
     # 2 pi-periodic and 1 + sin(theta/2) is symmetric about pi); the thresholds leave (0, 1/2]
     ["thresholds"]),
    ("extent without the square (Eq. 5)", EO,
     "xi *= (math.cos(a) + math.sin(a)) ** 2", "xi *= (math.cos(a) + math.sin(a))",
     ["extent_all_pi"]),
    ("e instead of e^2 in Eq. 6", EO,
     "math.log(2.0 * (math.e * math.e) / delta)", "math.log(2.0 * math.e / delta)",
     ["eq6_values", "eq6_limits"]),
    ("numerator of Eq. 6 not squared", EO,
     "num = (math.sqrt(xi) + math.sqrt(p_max)) ** 2", "num = (math.sqrt(xi) + math.sqrt(p_max))",
     ["eq6_values", "eq6_limits"]),
    ("flip probability cos/(sin + cos) instead of sin/(sin + cos) (Eq. 11)", EO,
     "p1 = sa / (sa + ca)", "p1 = ca / (sa + ca)",
     ["thresholds", "raw_unbiased"]),
    ("importance ratio without the factor i (Eq. 10)", EO,
     "np.where(X[:, j] == 1, 1j * ratio1[j], ratio0[j])", "np.where(X[:, j] == 1, ratio1[j], ratio0[j])",
     ["raw_unbiased", "raw_converges"]),
    ("importance ratio with p_T(x = 1) for x = 0 (Eq. 10)", EO,
     'cp["c"] / cp["pT0"]', 'cp["c"] / max(cp["pT1"], 1e-300)',
     ["raw_zero_angles", "raw_unbiased", "raw_converges"]),
    ("standard error without the factor 2 (delta method for |alpha|^2)", EO,
     "stderr[i] = 2.0 * math.sqrt(", "stderr[i] = 1.0 * math.sqrt(",
     ["stderr_spread"]),
    ("standard error twice too large", EO,
     "stderr[i] = 2.0 * math.sqrt(", "stderr[i] = 4.0 * math.sqrt(",
     ["stderr_spread"]),
    ("p_hat as the mean of |Y|^2 instead of |mean Y|^2 (Section III-A)", EO,
     "p_hat[i] = abs(a) ** 2", "p_hat[i] = float(np.mean(np.abs(Y) ** 2))",
     ["raw_unbiased", "raw_converges"]),
    ("branch weights and thresholds from the unwrapped angle", EO,
     'th = wrap_angle(float(g["theta"]))', 'th = float(g["theta"])',
     # Eq. 7 holds for every real theta, so Exact results cannot see this; the thresholds can
     ["thresholds"]),
    ("global phase e^{+i theta/4}", EO,
     "np.exp(-1j * sum(cp[\"theta\"] for cp in self.cps) / 4.0)",
     "np.exp(1j * sum(cp[\"theta\"] for cp in self.cps) / 4.0)",
     ["exact_vs_statevector", "lucj12"]),
    ("derivative of cos(theta/4) with the wrong sign", EO,
     '-cp["s"] / 4.0', 'cp["s"] / 4.0',
     ["fd_gradient", "sv_derivative"]),
    ("product rule without the segment's own derivative", EO,
     "dseg = dG @ seg + G @ dseg", "dseg = dG @ seg",
     ["fd_gradient", "sv_derivative"]),
    ("derivative of D_x with theta/4 instead of theta/2", EO,
     'dd_coef[:, cp["p"]] += 0.5j * v', 'dd_coef[:, cp["p"]] += 0.25j * v',
     # in the gradient pin's circuit a phase on those modes only changes the amplitude's phase:
     # the amplitude derivative sees it, the probability derivative cannot
     ["sv_derivative"]),
    ("determinant derivative keeping only the last column", EO,
     "out += np.linalg.det(Ai)", "out = np.linalg.det(Ai)",
     ["fd_gradient", "sv_derivative"]),
    ("derivative of the global phase with the wrong sign", EO,
     "dphase = -0.25j * sum(", "dphase = 0.25j * sum(",
     ["sv_derivative"]),
    ("Estimate rounds that never tighten p_max", EO,
     "pmax[i] = min(pmax[i], ph[i] + eps_r)", "pmax[i] = pmax[i]",
     ["estimate_eps"]),
    ("SplitMix64 multiplier off by one", EO,
     "0xBF58476D1CE4E5B9", "0xBF58476D1CE4E5B8",
     ["splitmix64"]),
    ("trajectory counts rounded down", EO,
     "m = -(-t // (1 << e))", "m = t // (1 << e)",
     ["trajectory_grid"]),
    ("Philox with nine rounds", PH,
     "for _ in range(10):", "for _ in range(9):",
     ["philox_kat"]),
    ("Philox mixing the wrong key word", PH,
     "hi1 ^ c1 ^ k0", "hi1 ^ c1 ^ k1",
     ["philox_kat"]),
]


def _param_list(fn):
    for m in getattr(fn, "pytestmark", []):
        if m.name == "parametrize":
            return m.args[1]
    raise LookupError(fn.__name__)


def _pins():
    """Each pin as a no-argument callable (parametrised pins run every case)."""
    def each(fn):
        cases = _param_list(fn)
        return lambda: [fn(*c) if isinstance(c, tuple) else fn(c) for c in cases]

    return {
        "philox_kat": PINS.test_philox_known_answer_vectors,
        "exact_vs_statevector": each(PINS.test_exact_amplitudes_match_statevector),
        "lucj12": PINS.test_exact_lucj_12_qubits_all_400_outcomes,
        "k0_minor": PINS.test_k0_is_a_single_minor_of_the_network_unitary,
        "cphase_identity": PINS.test_zero_angle_cphase_is_identity_and_angles_wrap,
        "extent_all_pi": PINS.test_extent_all_pi_is_two_to_the_k,
        "printed_extents": PINS.test_printed_extents_reproduce_under_the_variance_reading,
        "fig3": PINS.test_fig3_worked_example,
        "thresholds": PINS.test_thresholds_match_eq_10_11,
        "eq6_values": each(PINS.test_trajectory_bound_eq6_worked_values),
        "eq6_limits": PINS.test_trajectory_bound_eq6_limits_and_monotonicity,
        "splitmix64": PINS.test_splitmix64_known_answers,
        "trajectory_grid": PINS.test_trajectory_grid,
        "estimate_eps": PINS.test_estimate_oracle_meets_eps,
        "raw_zero_angles": PINS.test_raw_estimate_zero_angles_is_exact,
        "raw_unbiased": PINS.test_raw_estimate_unbiased_amplitude_and_exact_bias_formula,
        "raw_converges": PINS.test_raw_estimate_converges_and_stderr_is_calibrated,
        "stderr_spread": PINS.test_raw_estimate_stderr_matches_spread_over_seeds,
        "fd_gradient": PINS.test_forward_mode_gradient_matches_central_differences,
        "sv_derivative": PINS.test_forward_mode_derivative_of_amplitude_matches_statevector_differences,
    }


def _mutant_module(module, old, new):
    src = inspect.getsource(module)
    assert src.count(old) == 1, f"mutation site not unique or gone: {old!r}"
    m = types.ModuleType(module.__name__ + "_mutant")
    m.__package__ = "oracle"
    m.__file__ = module.__file__
    exec(compile(src.replace(old, new), module.__file__ + " (mutant)", "exec"), m.__dict__)
    return m


def mutant_oracle(module, old, new):
    """The oracle package's public names, with those defined in ``module``
    taken from its mutated copy (the state-vector reference stays intact)."""
    mut = _mutant_module(module, old, new)
    ns = types.SimpleNamespace(**{k: getattr(oracle, k) for k in dir(oracle) if not k.startswith("_")})
    for k in list(vars(ns)):
        if getattr(module, k, None) is getattr(oracle, k) and hasattr(mut, k):
            setattr(ns, k, getattr(mut, k))
    return ns


def pin_fails(name, ns, monkeypatch):
    with monkeypatch.context() as mp:
        mp.setattr(PINS, "O", ns)
        try:
            _pins()[name]()
        except Exception:  # an assertion, or the mutant breaking outright
            return True
    return False


def test_unmutated_oracle_passes_the_pins_used_here(monkeypatch):
    ns = types.SimpleNamespace(**{k: getattr(oracle, k) for k in dir(oracle) if not k.startswith("_")})
    used = sorted({p for *_, pins in MUTANTS for p in pins})
    assert [p for p in used if pin_fails(p, ns, monkeypatch)] == []


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # some mutants overflow, as expected
@pytest.mark.parametrize("name,module,old,new,catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, module, old, new, catchers, monkeypatch):
    ns = mutant_oracle(module, old, new)
    assert any(pin_fails(p, ns, monkeypatch) for p in catchers), f"no pin caught: {name}"
