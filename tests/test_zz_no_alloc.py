"""The allocation-free Exact entry point (ef_prob_exact_noalloc_dev).

Some callers cannot let a library allocate GPU memory while they run (their
memory is handed to their own pool at start-up, or a cudaMalloc/cudaFree
would synchronise the device in a latency-bound loop). For them the library
offers an Exact entry point whose scratch lives in a fixed per-GPU array.
These tests call it through the C ABI, twice in a row on the shared array,
and compare with the ordinary entry point within the tolerances the other
GPU tests use. This file is collected last on purpose."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _floor(c):
    meta = c.meta
    if "norb" in meta:
        return 1e-6 / (math.comb(meta["norb"], meta["n_alpha"]) * math.comb(meta["norb"], meta["n_beta"]))
    return 1e-6 / math.comb(c.n_modes, len(c.occupied_modes()))


CASES = [
    ("brick8_exact", lambda: W.brick8_exact()),
    ("lucj-12q", lambda: (W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3,
                                         angle_sampler=W.normal_var(0.1, math.pi), seed=7),
                          W.spin_sector_bitstrings_all(6, 3, 3))),
    ("lucj-32q-1500", lambda: W.lucj32_exact(1500)),
]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("auto", 1e-5)])
def test_noalloc_matches_allocating_entry_point_twice(lib, name, maker, prec, tol):
    c, bits = maker()
    precision = {"fp64": lib.EF_PREC_FP64, "fp32": lib.EF_PREC_FP32_MINOR, "auto": lib.EF_PREC_AUTO}[prec]
    nb = len(bits)
    d_bits = torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).cuda()
    ref = torch.empty(nb, dtype=torch.float64, device="cuda")
    out = torch.empty(nb, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    h_ref = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=precision)
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=precision)
    try:
        lib.ef_prob_exact_dev(h_ref, d_bits.data_ptr(), nb, ref.data_ptr(), 0, stream.cuda_stream)
        for _ in range(2):
            out.fill_(-1.0)
            lib.ef_prob_exact_noalloc_dev(h, d_bits.data_ptr(), nb, out.data_ptr(), 0, stream.cuda_stream)
            stream.synchronize()
            p, p_ref = out.cpu().numpy(), ref.cpu().numpy()
            assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, _floor(c))) <= tol
    finally:
        lib.ef_circuit_destroy(h)
        lib.ef_circuit_destroy(h_ref)


def test_noalloc_alternating_circuits(lib):
    """Two circuits in turn on the shared array: each call after the other
    circuit's copies its own tables in again; a repeated call on the same
    circuit finds them in place. Every result equals the allocating entry
    point's."""
    cases = [CASES[0][1](), CASES[1][1]()]
    stream = torch.cuda.current_stream()
    hs, refs, devs = [], [], []
    try:
        for c, bits in cases:
            h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO)
            hs.append(h)
            d_bits = torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).cuda()
            ref = torch.empty(len(bits), dtype=torch.float64, device="cuda")
            lib.ef_prob_exact_dev(h, d_bits.data_ptr(), len(bits), ref.data_ptr(), 0, stream.cuda_stream)
            devs.append(d_bits)
            refs.append(ref)
        for i in (0, 1, 1, 0, 1):
            out = torch.full((len(cases[i][1]),), -1.0, dtype=torch.float64, device="cuda")
            lib.ef_prob_exact_noalloc_dev(hs[i], devs[i].data_ptr(), len(cases[i][1]), out.data_ptr(), 0,
                                          stream.cuda_stream)
            stream.synchronize()
            p, p_ref = out.cpu().numpy(), refs[i].cpu().numpy()
            assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, _floor(cases[i][0]))) <= 1e-5
    finally:
        for h in hs:
            lib.ef_circuit_destroy(h)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch(lib):
    c, _ = W.lucj32_exact(0)
    nb = 200_000
    # real buffers of the full size, so that the call would be valid if it ran
    bits = W.spin_sector_bitstrings(16, 8, 8, 64, np.random.default_rng(0))
    d_bits = torch.from_numpy(np.tile(bits, (nb // 64, 1)).view(np.int64)).cuda()
    out = torch.zeros(nb, dtype=torch.float64, device="cuda")
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates)
    try:
        with pytest.raises(lib.ExtraFermError) as e:
            lib.ef_prob_exact_noalloc_dev(h, d_bits.data_ptr(), nb, out.data_ptr(), 0,
                                          torch.cuda.current_stream().cuda_stream)
        assert e.value.status == lib.EF_EINVAL
        assert "at most" in str(e.value)
        assert float(out.abs().max()) == 0.0
    finally:
        lib.ef_circuit_destroy(h)


def test_noalloc_call_captured_in_a_cuda_graph(lib):
    """Once a call has put the circuit's tables in the fixed array, the next
    call on the same circuit and stream copies nothing, synchronises nothing
    and allocates nothing, so it can be captured in a CUDA graph; the
    replayed graph gives the allocating entry point's results."""
    c, bits = W.lucj32_exact(1500)
    nb = len(bits)
    d_bits = torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).cuda()
    ref = torch.empty(nb, dtype=torch.float64, device="cuda")
    out = torch.full((nb,), -1.0, dtype=torch.float64, device="cuda")
    h_ref = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO)
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO)
    s = torch.cuda.Stream()
    try:
        lib.ef_prob_exact_dev(h_ref, d_bits.data_ptr(), nb, ref.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            lib.ef_prob_exact_noalloc_dev(h, d_bits.data_ptr(), nb, out.data_ptr(), 0, s.cuda_stream)
        s.synchronize()
        out.fill_(-1.0)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            lib.ef_prob_exact_noalloc_dev(h, d_bits.data_ptr(), nb, out.data_ptr(), 0, s.cuda_stream)
        for _ in range(2):
            g.replay()
            torch.cuda.synchronize()
            p, p_ref = out.cpu().numpy(), ref.cpu().numpy()
            assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, _floor(c))) <= 1e-5
            out.fill_(-1.0)
    finally:
        lib.ef_circuit_destroy(h)
        lib.ef_circuit_destroy(h_ref)
