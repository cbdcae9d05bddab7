"""The bench's reference arm on CPU: `bench.py --impl reference` times the FP64
oracle on the host cores and prints one JSON line with the same metric, unit
and workload as the CUDA arm; under a multi-rank launch only rank 0 works.
Also the host logic of the CUDA arm's Estimate sub-object, with a stand-in
for the binding."""
import json
import math
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run(extra_env=None, timeout=600):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def _json_lines(stdout):
    out = []
    for line in stdout.splitlines():
        line = line.strip()
        if line.startswith("{"):
            out.append(json.loads(line))
    return out


def test_reference_arm_prints_one_contract_line():
    import bench
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    # same metric, unit, direction and workload as the CUDA arm
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["n_gpus"] == 1 and d["steps"] == 1
    assert d["warmup"] == 3  # warm-up is raised to at least 3 steps
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["cores"], int) and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the line's throughput is the sampled bitstrings over the timed wall time
    per_step = int(cb["sample"].split()[0])
    assert abs(d["value"] - per_step / (d["ms_per_step"] / 1e3)) <= 1e-9 * d["value"]


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert _json_lines(r.stdout) == []


def test_estimate_sub_object_shape_with_a_stand_in_binding():
    """The Estimate sub-object's host logic (no GPU): a stand-in for the
    binding returns fixed trajectory counts; the sub-object reports them with
    the Eq. 6 count of one Raw Estimate at p_max = 1 beside them."""
    import numpy as np

    import bench

    class StandIn:
        EF_PREC_AUTO = 2

        def ef_circuit_create(self, n, occ, gates, precision=0, tol=0.0):
            return object()

        def ef_circuit_extent(self, h):
            return 4.0

        def ef_prob_estimate(self, h, bits, eps, delta, seed=0, index_base=0):
            n = len(bits)
            return np.zeros(n), np.zeros(n), np.full(n, 1000, dtype=np.int64)

        def ef_circuit_destroy(self, h):
            pass

    d = bench.bench_estimate(StandIn(), n_bits=50)
    assert d["unit"] == bench.UNIT and d["value"] > 0 and d["steps"] == 2
    assert d["trajectories_per_bitstring_mean"] == 1000 and d["trajectories_per_bitstring_max"] == 1000
    # Eq. 6 at p_max = 1, eps = delta = 0.01, extent 4: 2 (2 + 1)^2 / (sqrt(1.01) - 1)^2 log(2 e^2 / 0.01)
    want = math.ceil(2 * 9 / (math.sqrt(1.01) - 1) ** 2 * math.log(2 * math.e ** 2 / 0.01))
    assert d["one_shot_eq6_at_pmax_1"] == want
