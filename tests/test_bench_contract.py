"""bench.py without a GPU: the reference arm's JSON line, its behaviour under torchrun with
two ranks, and the multi-rank aggregation of the GPU arm (max over ranks, whole-job rate)
on world-size-2 gloo process groups.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.strip().startswith("{")]


# the 12-site ring keeps the reference arm's full oracle step short on this host
REF_ARGS = ["--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-rows", "2000",
            "--workload", "ring12_3_3"]


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", *REF_ARGS], cwd=ROOT, capture_output=True,
                         text=True, timeout=300, check=True)
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["ms_per_step"] == pytest.approx(1e3 / d["value"])
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # measured on one full oracle step; the same config dict as the GPU arm's
    assert d["full_step_s"] > 0 and d["value"] == pytest.approx(1.0 / d["full_step_s"])
    assert d["config"] == bench._workload_config("ring12_3_3")
    assert d["config"]["dim"] == 220 * 220


def test_reference_values_come_from_stored_oracle_results():
    E, src = bench.reference_E0("torus4x4_5_5", 4.0)
    assert E == pytest.approx(-19.5809375254, abs=1e-9) and "oracle" in src
    E, src = bench.reference_E0("ring16_8_8", 4.0)
    assert E == pytest.approx(-9.21443097198, abs=1e-9) and "Bethe" in src
    assert len(bench.golden_batched()) == 256


def test_reference_arm_two_ranks_prints_once():
    """Under torchrun only rank 0 runs the oracle and prints; the other rank exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--gpus", "2", *REF_ARGS]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


_WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=ws)
# each rank's own step time and H.v time (ms); the slowest rank decides
mine = [10.0 + 5.0 * rank, 7.0 - rank]
got = bench._max_over_ranks(mine, "cpu")
rate = bench._whole_job_rate(ws, 100, got[0] / 1e3)
print(json.dumps({"rank": rank, "max": got, "rate": rate}), flush=True)
dist.destroy_process_group()
"""


def test_max_over_ranks_gloo_world_size_2():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    res = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e[-2000:]
        res.append(_json_lines(o)[0])
    for r in res:
        assert r["max"] == [15.0, 7.0]  # element-wise max over the two ranks
        assert r["rate"] == pytest.approx(2 * 100 / 0.015)  # units of both ranks / slowest time


def test_single_process_aggregation_is_identity():
    assert bench._max_over_ranks([3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench._whole_job_rate(1, 50, 0.5) == 100.0
