"""Multi-circuit batch (ef_batch_*): one planned, graph-captured execution
of circuits of uneven modes, particles and controlled-phase counts must give
the same results as the circuits' own calls (the same kernels compute every
minor the same way, so the results are identical), on the first call, on the
graph replay and after a change of angles; and agree with the oracle."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _small_batch():
    rng = np.random.default_rng(8)
    out = []
    out.append((W.brick8_exact()[0], W.brick8_exact()[1], 0))
    out.append((W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1), seed=7),
                W.spin_sector_bitstrings_all(6, 3, 3), 0))
    out.append((W.lucj_circuit(5, 2, 2, 2, n_onsite=3, n_same=2, angle_sampler=W.normal_var(0.5), seed=8),
                W.spin_sector_bitstrings_all(5, 2, 2), 0))
    out.append((W.random_fig4_circuit(10, 5, 6, 3, seed=22), W.sector_bitstrings(10, 5, 333, rng), 0))
    out.append((W.lucj_circuit(8, 3, 3, 1, n_onsite=8, n_same=3, angle_sampler=W.normal_var(0.1), seed=9),
                W.spin_sector_bitstrings(8, 3, 3, 1000, rng), 0))
    out.append((W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1), seed=17),
                W.spin_sector_bitstrings_all(6, 3, 3)[:57], 300))
    out.append((W.random_fig4_circuit(10, 4, 7, 3, seed=31, angle_std=1.2), W.sector_bitstrings_all(10, 4)[:60], 500))
    out.append((W.lucj_circuit(10, 9, 9, 1, n_onsite=4, n_same=2, angle_sampler=W.normal_var(0.1), seed=19),
                W.spin_sector_bitstrings(10, 9, 9, 20, rng), 200))
    return out


def _dev(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).cuda()


def test_batch_equals_individual_calls_and_replays(lib):
    items = _small_batch()
    hs = [lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO) for c, _, _ in items]
    b = lib.ef_batch_create(hs)
    try:
        dbits = [_dev(bits) for _, bits, _ in items]
        outs = [torch.full((len(bits),), -1.0, dtype=torch.float64, device="cuda") for _, bits, _ in items]
        nb = [len(bits) for _, bits, _ in items]
        traj = [t for _, _, t in items]
        stream = torch.cuda.current_stream()
        refs = []
        for h, (c, bits, t) in zip(hs, items):
            refs.append(lib.ef_prob_exact(h, bits) if t == 0 else lib.ef_prob_approx(h, bits, t, seed=5)[0])
        for call in range(3):
            for o in outs:
                o.fill_(-1.0)
            lib.ef_batch_prob_dev(b, [d.data_ptr() for d in dbits], nb, [o.data_ptr() for o in outs], traj, 5,
                                  stream.cuda_stream)
            stream.synchronize()
            for o, ref in zip(outs, refs):
                assert np.array_equal(o.cpu().numpy(), ref), call
        st = lib.ef_batch_get_stats(b)
        assert st["kernel_launches"] > 0
        # a change of angles re-plans and still matches
        c0 = items[1][0]
        ang = O.get_angles(c0.gates) * 0.9
        lib.ef_circuit_set_angles(hs[1], ang)
        lib.ef_batch_prob_dev(b, [d.data_ptr() for d in dbits], nb, [o.data_ptr() for o in outs], traj, 5,
                              stream.cuda_stream)
        stream.synchronize()
        assert np.array_equal(outs[1].cpu().numpy(), lib.ef_prob_exact(hs[1], items[1][1]))
        c1 = W.Circuit(c0.n_modes, c0.occupation, O.set_angles(c0.gates, ang), meta=c0.meta)
        p_ref = O.exact_probabilities(c1, items[1][1])
        floor = 1e-6 / 400
        assert np.max(np.abs(outs[1].cpu().numpy() - p_ref) / np.maximum(p_ref, floor)) <= 1e-5
    finally:
        lib.ef_batch_destroy(b)
        for h in hs:
            lib.ef_circuit_destroy(h)


def test_batch_uneven64_subset(lib):
    """The 64 uneven circuits of the batch workload, 300 bitstrings each and
    200 trajectories for the approximate ones: the batch matches the
    individual calls, and the oracle on sampled exact results."""
    batch = W.uneven_batch64()
    hs, dbits, outs, nb, traj = [], [], [], [], []
    for c, bits, mode in batch:
        hs.append(lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO))
        sub = bits[:300]
        dbits.append(_dev(sub))
        outs.append(torch.zeros(len(sub), dtype=torch.float64, device="cuda"))
        nb.append(len(sub))
        traj.append(0 if mode == "exact" else 200)
    b = lib.ef_batch_create(hs)
    try:
        stream = torch.cuda.current_stream()
        lib.ef_batch_prob_dev(b, [d.data_ptr() for d in dbits], nb, [o.data_ptr() for o in outs], traj, 3,
                              stream.cuda_stream)
        stream.synchronize()
        checked = 0
        for i, (c, bits, mode) in enumerate(batch):
            sub = bits[:300]
            ref = lib.ef_prob_exact(hs[i], sub) if mode == "exact" else lib.ef_prob_approx(hs[i], sub, 200, seed=3)[0]
            assert np.array_equal(outs[i].cpu().numpy(), ref), i
            if mode == "exact" and c.n_cphase <= 10 and c.n_modes <= 24 and checked < 3:
                norb = c.n_modes // 2
                eta = len(c.occupied_modes()) // 2
                p_ref = O.exact_probabilities(c, sub[:4])
                floor = 1e-6 / math.comb(norb, eta) ** 2
                assert np.max(np.abs(ref[:4] - p_ref) / np.maximum(p_ref, floor)) <= 1e-5
                checked += 1
        assert checked >= 1
    finally:
        lib.ef_batch_destroy(b)
        for h in hs:
            lib.ef_circuit_destroy(h)


def test_batch_rejects_a_circuit_listed_twice(lib):
    c, _ = W.brick8_exact()
    h = lib.ef_circuit_create(c.n_modes, c.occupation, c.gates)
    try:
        with pytest.raises(lib.ExtraFermError) as e:
            lib.ef_batch_create([h, h])
        assert e.value.status == lib.EF_EINVAL
    finally:
        lib.ef_circuit_destroy(h)


def test_batch_replans_after_a_direct_call_regrows_a_workspace(lib):
    """The captured graph holds the circuits' workspace addresses. A direct
    call with many more bitstrings reallocates circuit 0's determinant
    buffers; the next batch call must re-plan (not replay stale addresses)
    and still give the circuits' own results."""
    rng = np.random.default_rng(4)
    items = [(W.lucj_circuit(6, 3, 3, 1, n_onsite=6, n_same=3, angle_sampler=W.normal_var(0.1), seed=7),
              W.spin_sector_bitstrings_all(6, 3, 3)[:40], 0),
             (W.random_fig4_circuit(10, 4, 7, 3, seed=31, angle_std=1.2), W.sector_bitstrings_all(10, 4)[:30], 300)]
    hs = [lib.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=lib.EF_PREC_AUTO) for c, _, _ in items]
    b = lib.ef_batch_create(hs)
    try:
        dbits = [_dev(bits) for _, bits, _ in items]
        outs = [torch.zeros(len(bits), dtype=torch.float64, device="cuda") for _, bits, _ in items]
        nb = [len(bits) for _, bits, _ in items]
        traj = [t for _, _, t in items]
        stream = torch.cuda.current_stream()

        def run():
            for o in outs:
                o.fill_(-1.0)
            lib.ef_batch_prob_dev(b, [d.data_ptr() for d in dbits], nb, [o.data_ptr() for o in outs], traj, 9,
                                  stream.cuda_stream)
            stream.synchronize()
            return [o.cpu().numpy() for o in outs]

        first = run()
        again = run()  # replay
        many = W.spin_sector_bitstrings(6, 3, 3, 20_000, rng)
        lib.ef_prob_exact(hs[0], many)  # regrows circuit 0's workspace
        lib.ef_prob_approx(hs[1], W.sector_bitstrings(10, 4, 5_000, rng), 50)  # and circuit 1's partial sums
        after = run()
        refs = [lib.ef_prob_exact(hs[0], items[0][1]), lib.ef_prob_approx(hs[1], items[1][1], 300, seed=9)[0]]
        for i in range(2):
            assert np.array_equal(first[i], refs[i]) and np.array_equal(again[i], refs[i])
            assert np.array_equal(after[i], refs[i])
    finally:
        lib.ef_batch_destroy(b)
        for h in hs:
            lib.ef_circuit_destroy(h)
