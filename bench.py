#!/usr/bin/env python
"""Throughput benchmark of the Exact probability path on the LUCJ-shaped
workload: 32 qubits (2x16 spin-orbital modes), 8 alpha + 8 beta electrons,
one Jastrow layer of k=16 controlled-phase gates (4 aa + 4 bb nearest
neighbour, 8 ab on-site, angles N(0, 0.1)) between a Haar orbital rotation
and its inverse; 2^16 branches; 10^4 bitstrings uniform in the (8,8) sector.

One step = one ef_prob_exact_dev call on device-resident bitstrings: branch
matrices, FP32 minor LUs, FP64 branch sums, per-result error estimate and
the FP64 recomputation of flagged results (EF_PREC_AUTO, tol 1e-5).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica on its own 10^4 bitstrings
(weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "Born-rule probabilities/s and branch-dets/s at rel err ≤1e-5 vs FP64 oracle"
UNIT = "probabilities/s"
NB = 10_000
# dram__bytes_read.sum + dram__bytes_write.sum of one k_exact_lu_f32<8> launch on this workload
# (ncu, GB300, `-k regex:"k_exact_lu_f32|k_exact_combine_wp" -s 9 -c 6` on `bench.py --steps 3
# --warmup 3 --no-cpu-baseline --no-fp64-form`): one launch covers both mode blocks; of the 82 MB of FP32 determinants it
# writes, 24-27 MB reach DRAM within the launch and the rest stays in L2 until the combine; the
# pattern matrices are read from L2. To be re-measured whenever that kernel changes.
LU_DRAM_BYTES_PER_LAUNCH = 26_846_848  # mean of two launches (28.4 MB, 25.3 MB), 8-pattern chunks
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flops x max SM clock
L2_BYTES = 129 * 2 ** 20
BATCH_TRAJ = 1000  # trajectories per Raw Estimate circuit of the batch workload
WORKLOAD = ("LUCJ exact: 2x16 modes (32 qubits), 8a+8b, k=16 controlled-phase gates "
            "(4 aa + 4 bb neighbour, 8 ab on-site, N(0,0.1)), 2^16 branches, 10^4 sector bitstrings")


# ----------------------------------------------------------------------------- oracle workers (CPU)

_ORACLE_CACHE = {}


def _oracle_worker(task):
    """Run the FP64 CPU oracle on bitstrings ``idx`` of the workload's batch
    ``seed_rank``; returns (seconds, probabilities)."""
    idx, rank = task
    import oracle as O
    key = ("c2", rank)
    if key not in _ORACLE_CACHE:
        c, bits = make_workload(rank)
        _ORACLE_CACHE[key] = (c, bits)
    c, bits = _ORACLE_CACHE[key]
    t0 = time.perf_counter()
    p = O.exact_probabilities(c, bits[np.asarray(idx, dtype=np.int64)])
    return time.perf_counter() - t0, p.tolist()


def make_workload(rank: int = 0):
    c, _ = W.lucj32_exact(0)
    rng = np.random.default_rng(replica_plan(rank, 1, NB)[0])
    bits = W.spin_sector_bitstrings(16, 8, 8, NB, rng)
    return c, bits


def oracle_pool(ncores):
    import multiprocessing as mp
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(ncores)
    pool.map(_oracle_worker, [([0], 0)] * ncores)  # import and cache in every worker
    return pool


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(pool, ncores, per_core, offset=0, rank=0):
    """Wall time of the oracle on ncores * per_core bitstrings, spread over the pool."""
    tasks = [(list(range(offset + i * per_core, offset + (i + 1) * per_core)), rank) for i in range(ncores)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, tasks)
    wall = time.perf_counter() - t0
    idx = [j for t in tasks for j in t[0]]
    p = np.array([v for r in res for v in r[1]])
    return wall, idx, p


# ----------------------------------------------------------------------------- clocks


def start_clock_sampler(path, gpu_index):
    if shutil.which("nvidia-smi") is None:
        return None
    q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    f = open(path, "w")
    p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}", "--format=csv,noheader",
                          "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
    return p, f


def stop_clock_sampler(handle, path, t_begin, t_end):
    if handle is None:
        return None
    p, f = handle
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    f.close()
    rows = []
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
            sm = float(parts[2].split()[0])
            smax = float(parts[3].split()[0])
        except (ValueError, IndexError):
            continue
        rows.append((ts, sm, smax, parts[6:10]))
    if not rows:
        return None
    sel = [r for r in rows if t_begin - 1 <= r[0] <= t_end + 1] or rows
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in sel for i, v in enumerate(r[3]) if v.lower() == "active"})
    return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
            "reasons": reasons, "samples": len(sel)}


# ----------------------------------------------------------------------------- arms


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_plan(rank: int, world: int, nb: int):
    """Replicas only: rank r evaluates its own batch of nb bitstrings (seeded by r)
    whose global indices start at r * nb, so Raw Estimate trajectories never repeat
    across ranks. Returns (bitstring seed, global index base)."""
    return 1002 + 7919 * rank, rank * nb


def aggregate_timing(local_ms: float, world: int, nb: int, steps: int, dist=None) -> tuple[float, float]:
    """Whole-job throughput from the slowest rank: (max device ms over ranks,
    bitstrings of all ranks per second)."""
    worst = local_ms
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([local_ms], dtype=torch.float64)
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        worst = float(t.item())
    return worst, world * nb * steps / (worst / 1e3)


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    ncores = host_cores()
    pool = oracle_pool(ncores)
    per_core = 1
    times = []
    for s in range(args.warmup + args.steps):
        wall, _, _ = time_oracle(pool, ncores, per_core, offset=(s * ncores) % (NB - ncores))
        if s >= args.warmup:
            times.append(wall)
    pool.close()
    per_step = ncores * per_core
    value = per_step * len(times) / sum(times)
    sample = f"{per_step} bitstrings of the 10^4 per step ({per_core} per core), FP64 numpy oracle"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle": "plain FP64 CPU oracle (numpy), one process per core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_fp64_form(ef, torch, c, d_bits, p_gpu, flush, stream, dev, steps):
    """Device time of the EF_PREC_FP64 single-circuit form on the same bitstrings
    and the largest relative difference of the headline results from it."""
    h64 = ef.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=ef.EF_PREC_FP64)
    d_out64 = torch.empty(NB, dtype=torch.float64, device=dev)
    steps64 = min(steps, 5)
    ms64 = []
    for i in range(1 + steps64):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ef.ef_prob_exact_dev(h64, d_bits.data_ptr(), NB, d_out64.data_ptr(), 0, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if i >= 1:
            ms64.append(e0.elapsed_time(e1))
    ef.ef_circuit_destroy(h64)
    p64 = d_out64.cpu().numpy()
    floor64 = 1e-6 / math.comb(16, 8) ** 2
    return {"value": NB / (statistics.mean(ms64) / 1e3), "unit": UNIT, "ms_per_step": statistics.mean(ms64),
            "steps": steps64, "form": "EF_PREC_FP64 single circuit, same bitstrings, L2 flushed",
            "max_rel_diff_of_value_results": float(np.max(np.abs(p_gpu - p64) / np.maximum(p64, floor64)))}


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    pool = None
    ncores = host_cores()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(ncores)  # spawned before the first CUDA call

    import paper_2511_12416_gb300 as ef
    ef.load()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    c, bits = make_workload(rank)
    prec = {"auto": ef.EF_PREC_AUTO, "fp64": ef.EF_PREC_FP64, "fp32": ef.EF_PREC_FP32_MINOR}[args.precision]
    h = ef.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=prec, tol=1e-5,
                             flags=ef.EF_FLAG_TIME_KERNELS)
    d_bits = torch.from_numpy(bits.view(np.int64)).to(dev)
    d_out = torch.empty(NB, dtype=torch.float64, device=dev)
    d_err = torch.empty(NB, dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ef.ef_prob_exact_dev(h, d_bits.data_ptr(), NB, d_out.data_ptr(), d_err.data_ptr(), stream.cuda_stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    clk_path = os.path.join(tempfile.gettempdir(), f"ef_clocks_{os.getpid()}.csv")
    sampler = start_clock_sampler(clk_path, dev.index) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t_begin = time.time()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms = 0.0
    kern_launches = 0
    kern_flops = 0.0
    launches = 0
    recomputed = 0
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed steps, outside the step's events
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
        st = ef.ef_circuit_get_stats(h)
        kern_ms += st["dominant_kernel_ms"]
        kern_launches += st["dominant_kernel_launches"]
        kern_flops += st["dominant_kernel_flops"]
        launches += st["kernel_launches"]
        recomputed += st["fp64_recomputed"]
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t_end = time.time()
    clocks = stop_clock_sampler(sampler, clk_path, t_begin, t_end) if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms, value = aggregate_timing(sum(step_ms), world, NB, args.steps,
                                       torch.distributed if world > 1 else None)
    branch_dets = value * 2 ** 16
    last = ef.ef_circuit_get_stats(h)
    p_gpu = d_out.cpu().numpy()

    # end to end through the host API: pinned host buffers, H2D and D2H inside the timed region
    hb = torch.from_numpy(bits.view(np.int64)).pin_memory()
    e2e_bits = hb.numpy().view(np.uint64)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = ef.ef_prob_exact(h, e2e_bits)
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = NB / statistics.mean(e2e_times)
    if world > 1:
        tt = torch.tensor([e2e_value], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MIN)
        e2e_value = float(tt.item()) * world
    assert np.array_equal(out, p_gpu)

    cpu = None
    if pool is not None:
        per_core = max(1, int(math.ceil(64 / ncores)))
        wall, idx, p_ref = time_oracle(pool, ncores, per_core)
        pool.close()
        floor = 1e-6 / math.comb(16, 8) ** 2
        max_rel = float(np.max(np.abs(p_gpu[idx] - p_ref) / np.maximum(p_ref, floor)))
        cpu = {"value": len(idx) / wall, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": f"{len(idx)} of the 10^4 bitstrings ({per_core} per core), FP64 numpy oracle, "
                         f"one process per core; max rel err of the GPU results on them {max_rel:.2e}"}

    # the plain FP64 single-circuit form on the same bitstrings (minors, LU and sums in FP64)
    fp64_form = None
    if not args.no_fp64_form:
        fp64_form = time_fp64_form(ef, torch, c, d_bits, p_gpu, flush, stream, dev, args.steps)

    kern_s = kern_ms / 1e3
    achieved = kern_flops / kern_s / 1e12 if kern_s > 0 else 0.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "bitstrings_per_gpu": NB, "precision": args.precision,
                   "arithmetic": "FP32 minors and LU, float-pair (~48-bit) branch sums, FP64 redo of the "
                                 "determinants that carry a flagged result's estimated error",
                   "l2": "flushed between timed steps (2x L2 buffer written outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "branch_dets_per_s": branch_dets,
        "executed_lus_per_step": last["executed_minor_lus"],
        "fp64_recomputed_per_step": recomputed / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": LU_DRAM_BYTES_PER_LAUNCH,
                     "kernel": "k_exact_lu_f32 (FP32 LU of the per-block minors)",
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"},
        "dominant_kernel_ms_per_step": kern_ms / args.steps,
        "fp64_single_circuit": fp64_form,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": NB * 16, "d2h_bytes_per_step": NB * 8},
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    ef.ef_circuit_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0



# ----------------------------------------------------------------------------- secondary workloads
# (`--workload approx|grad|batch`): one JSON line each, device time with CUDA events, L2 flushed
# between steps; the default run measures the Exact workload above.


def _timed_steps(torch, dev, stream, flush, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    return ms


def run_secondary(args):
    import torch
    import paper_2511_12416_gb300 as ef

    ef.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "workload_kind": args.workload}
    launches = 0
    if args.workload == "approx":
        c, bits = W.lucj52_approx(args.nb)
        h = ef.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=ef.EF_PREC_FP32_MINOR)
        t = W.lucj52_trajectories(ef.ef_circuit_extent(h))
        d_bits = torch.from_numpy(bits.view(np.int64)).to(dev)
        d_out = torch.empty(len(bits), dtype=torch.float64, device=dev)
        d_se = torch.empty(len(bits), dtype=torch.float64, device=dev)
        seed = [0]

        def fn():
            seed[0] += 1
            ef.ef_prob_approx_dev(h, d_bits.data_ptr(), len(bits), t, seed[0], 0, d_out.data_ptr(),
                                  d_se.data_ptr(), stream.cuda_stream)
        ms = _timed_steps(torch, dev, stream, flush, fn, args.steps, args.warmup)
        launches = ef.ef_circuit_get_stats(h)["kernel_launches"]
        ef.ef_circuit_destroy(h)
        per = statistics.mean(ms)
        line.update({"metric": "Raw Estimate probabilities/s (FP32 minors, FP64 trajectory sums)",
                     "value": len(bits) / (per / 1e3), "unit": "probabilities/s", "ms_per_step": per,
                     "dtype": "f32",
                     "trajectories_per_s": len(bits) * t / (per / 1e3),
                     "config": {"workload": f"LUCJ 52-qubit approximate: 2x26 modes, 5a+5b, 2 layers, k=152, "
                                            f"t = ceil(extent/1e-4) = {t} trajectories per bitstring, "
                                            f"{len(bits)} of the 10^5 sector bitstrings per step",
                                "l2": "flushed between timed steps"}})
    elif args.workload == "grad":
        c, bits, w = W.lucj40_grad()
        h = ef.ef_circuit_create(c.n_modes, c.occupation, c.gates, precision=ef.EF_PREC_FP64)
        d_bits = torch.from_numpy(bits.view(np.int64)).to(dev)
        d_gp = torch.empty(len(bits), dtype=torch.float64, device=dev)
        d_p = torch.empty(len(bits), dtype=torch.float64, device=dev)
        d_g = torch.empty(ef.ef_circuit_num_angles(h), dtype=torch.float64, device=dev)
        ef.ef_prob_exact_dev(h, d_bits.data_ptr(), len(bits), d_p.data_ptr(), 0, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        # d/dp of sum_b w_b log p_b
        d_gp.copy_(torch.from_numpy(w).to(dev) / d_p.clamp_min(1e-300))

        def fn():
            ef.ef_prob_grad_dev(h, d_bits.data_ptr(), len(bits), d_gp.data_ptr(), d_p.data_ptr(), d_g.data_ptr(),
                                stream.cuda_stream)
        ms = _timed_steps(torch, dev, stream, flush, fn, args.steps, args.warmup)
        launches = ef.ef_circuit_get_stats(h)["kernel_launches"]
        n_ang = ef.ef_circuit_num_angles(h)
        ef.ef_circuit_destroy(h)
        per = statistics.mean(ms)
        line.update({"metric": "bitstring gradients/s (d p_b / d every angle, FP64 adjoint)",
                     "value": len(bits) / (per / 1e3), "unit": "bitstrings/s", "ms_per_step": per, "dtype": "f64",
                     "config": {"workload": f"LUCJ 40-qubit: 2x20 modes, 6a+6b, 2 layers, k=12, {len(bits)} "
                                            f"bitstrings, gradient of sum w_b log p_b w.r.t. {n_ang} angles",
                                "l2": "flushed between timed steps"}})
    else:  # batch
        batch = W.uneven_batch64()
        hs, dbits, outs, nb, traj = [], [], [], [], []
        for cc, bits, mode in batch:
            hs.append(ef.ef_circuit_create(cc.n_modes, cc.occupation, cc.gates, precision=ef.EF_PREC_AUTO))
            dbits.append(torch.from_numpy(bits.view(np.int64)).to(dev))
            outs.append(torch.empty(len(bits), dtype=torch.float64, device=dev))
            nb.append(len(bits))
            traj.append(0 if mode == "exact" else BATCH_TRAJ)
        b = ef.ef_batch_create(hs)
        ptr_b, ptr_o = [d.data_ptr() for d in dbits], [o.data_ptr() for o in outs]

        def fn():
            ef.ef_batch_prob_dev(b, ptr_b, nb, ptr_o, traj, 7, stream.cuda_stream)
        ms = _timed_steps(torch, dev, stream, flush, fn, args.steps, args.warmup)
        launches = ef.ef_batch_get_stats(b)["kernel_launches"]
        ef.ef_batch_destroy(b)
        for h in hs:
            ef.ef_circuit_destroy(h)
        per = statistics.mean(ms)
        n_exact = sum(1 for t in traj if t == 0)
        line.update({"metric": "probabilities/s over an uneven 64-circuit batch (one captured graph)",
                     "value": sum(nb) / (per / 1e3), "unit": "probabilities/s", "ms_per_step": per, "dtype": "f32",
                     "circuits_per_s": len(hs) / (per / 1e3),
                     "config": {"workload": f"64 circuits, n in 12..40, {sum(nb)} bitstrings, {n_exact} Exact "
                                            f"(EF_PREC_AUTO), {len(hs) - n_exact} Raw Estimate with {BATCH_TRAJ} "
                                            f"trajectories each; graph replay per step",
                                "l2": "flushed between timed steps"}})
    line["gpu_launches"] = launches
    print(json.dumps(line), flush=True)
    return 0


def main():
    global NB
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["auto", "fp64", "fp32"], default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip timing the FP64 single-circuit form")
    ap.add_argument("--nb", type=int, default=10_000, help="bitstrings per GPU (profiling runs use fewer)")
    ap.add_argument("--workload", choices=["exact", "approx", "grad", "batch"], default="exact",
                    help="exact: the headline line; the others measure the remaining paths, one line each")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    NB = args.nb
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "exact":
        return run_secondary(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
