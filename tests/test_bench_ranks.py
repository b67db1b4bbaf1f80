"""The multi-rank plumbing of bench.py on CPU: two gloo ranks, barrier and
max-over-ranks timing; the reference arm prints from rank 0 only."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import os, sys
sys.path.insert(0, %(root)r)
import bench
dist, world, rank, local = bench._dist_init()
assert world == 2 and dist is not None
bench._barrier(dist)
m = bench._max_over_ranks(dist, 1.5 + rank, "cpu")
print("RANK%%d MAX %%.2f" %% (rank, m))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_agree_on_max_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _CHILD % {"root": ROOT}], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    assert "RANK0 MAX 2.50" in outs[0][0]
    assert "RANK1 MAX 2.50" in outs[1][0]


def test_reference_arm_is_silent_off_rank0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    """`bench.py --impl reference` on rank 0: one JSON line with the base
    contract's keys, impl = reference, a cpu_baseline describing the run
    (kind, cores, sample; value equal to the line's), and an e2e entry with no
    host-device traffic."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--lattice", "8,8,8,8"], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
    # what was timed: ms_per_step is the measured sample (config.sweeps sweeps),
    # the whole-step figure only under its own, labelled key
    assert d["config"]["sweeps"] == 1 and d["config"]["lattice"] == [8, 8, 8, 8]
    assert abs(d["ms_per_step"] - cb["seconds"] * 1e3) < 1e-6 * d["ms_per_step"]
    assert d["extrapolated_ms_per_workload_step"]["sweeps"] == 300
