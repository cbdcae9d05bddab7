"""CPU-only checks of the C ABI: the library builds/loads, exports every
function include/extraferm.h declares, and its host preprocessing (argument
validation, angle layout, extent) agrees with the oracle. No probability is
computed here (that needs a GPU)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "extraferm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ef_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def ef():
    import paper_2511_12416_gb300 as ef
    ef.load()
    return ef


def test_library_exports_every_declared_symbol(ef):
    names = _declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(ef.lib_path())
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ef.SIGNATURES), "binding and header disagree"


def test_struct_layouts_match_header(ef):
    assert ctypes.sizeof(ef.EfGate) == 32
    assert ctypes.sizeof(ef.EfOptions) == 32
    assert ctypes.sizeof(ef.EfStats) == 72


def test_version_and_error_string(ef):
    assert ef.ef_version() >= 100
    with pytest.raises(ef.ExtraFermError) as e:
        ef.ef_circuit_create(0, [0, 0], W.make_gates([]))
    assert e.value.status == ef.EF_EINVAL
    assert "n_modes" in ef.ef_last_error()


@pytest.mark.parametrize("recs,occ,msg", [
    ([(W.GIVENS, 0, 2, 0.1, 0.2)], [0], "adjacent"),
    ([(W.GIVENS, 7, 8, 0.1, 0.2)], [0], "adjacent"),
    ([(W.CPHASE, 1, 1, 0.1, 0.0)], [0], "p != q"),
    ([(W.CPHASE, 1, 9, 0.1, 0.0)], [0], "p != q"),
    ([(W.PHASE, -1, 0, 0.0, 0.3)], [0], "out of range"),
    ([(7, 0, 1, 0.0, 0.0)], [0], "unknown"),
    ([(W.GIVENS, 0, 1, float("nan"), 0.0)], [0], "non-finite"),
    ([], [8], "occupation"),
])
def test_invalid_circuits_are_rejected(ef, recs, occ, msg):
    with pytest.raises(ef.ExtraFermError) as e:
        ef.ef_circuit_create(8, W.modes_to_bits(occ), W.make_gates(recs))
    assert e.value.status == ef.EF_EINVAL
    assert msg in str(e.value)


def test_angle_layout_and_extent_match_oracle(ef):
    for c in (W.brick8_exact()[0], W.lucj32_exact(16)[0], W.lucj52_approx(4)[0], W.lucj40_grad(8)[0]):
        h = ef.ef_circuit_create(c.n_modes, c.occupation, c.gates)
        try:
            assert np.array_equal(ef.ef_circuit_get_angles(h), O.get_angles(c.gates))
            assert math.isclose(ef.ef_circuit_extent(h), O.extent(c.gates), rel_tol=1e-13)
            a = O.get_angles(c.gates) + 0.25
            ef.ef_circuit_set_angles(h, a)
            assert np.array_equal(ef.ef_circuit_get_angles(h), a)
            assert math.isclose(ef.ef_circuit_extent(h), O.extent(O.set_angles(c.gates, a)), rel_tol=1e-13)
            with pytest.raises(ef.ExtraFermError):
                ef.ef_circuit_set_angles(h, a[:-1])
        finally:
            ef.ef_circuit_destroy(h)


def test_destroy_null_is_ok(ef):
    ef.load().ef_circuit_destroy(None)


def test_missing_library_raises(ef, tmp_path):
    """No CPU fallback: loading a library that is not there raises."""
    import subprocess
    import sys
    missing = str(tmp_path / "libextraferm.so")
    code = ("import paper_2511_12416_gb300 as ef\n"
            f"try:\n    ef.load({missing!r})\nexcept OSError:\n    print('raised')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "raised"


def test_product_code_does_not_reach_the_oracle():
    """The library, its binding and the input generators neither import nor
    name the oracle package (only the tests, smoke() and the bench's CPU legs
    may)."""
    pat = re.compile(r"^\s*(?:from\s+oracle\b|import\s+oracle\b)|extraferm_oracle|[\'\"]oracle[\'\"]", re.M)
    offenders = []
    for sub in ("paper_2511_12416_gb300", "workloads", "include"):
        for dirpath, _dirs, files in os.walk(os.path.join(ROOT, sub)):
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                    p = os.path.join(dirpath, f)
                    if pat.search(open(p, encoding="utf-8").read()):
                        offenders.append(os.path.relpath(p, ROOT))
    assert offenders == []


def test_oracle_does_not_reach_the_library():
    """The oracle is independent of the CUDA path: it neither imports the
    package nor loads its shared library."""
    pat = re.compile(r"paper_2511_12416_gb300|libextraferm|ctypes", re.M)
    offenders = []
    for dirpath, _dirs, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith((".py", ".c", ".h")):
                p = os.path.join(dirpath, f)
                if pat.search(open(p, encoding="utf-8").read()):
                    offenders.append(os.path.relpath(p, ROOT))
    assert offenders == []
