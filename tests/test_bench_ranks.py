"""The multi-rank side of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank of `bench.py --gpus N` solves its own replica; the only exchange is
host-side (a barrier, the maximum step time and the summed work over ranks),
and the reference arm runs on rank 0 alone.  These tests run those helpers in
two real processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import bench
rank, ws, dist = bench.dist_setup()
t = 1.0 + rank            # per-rank step time
w = 10.0 * (rank + 1)     # per-rank work
out = {"rank": rank, "ws": ws, "max": bench.dist_max(t, dist), "sum": bench.dist_sum(w, dist)}
dist.barrier()
dist.destroy_process_group()
print("RESULT " + json.dumps(out), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, ws=2, extra_env=None, timeout=120):
    port = _free_port()
    procs = []
    for r in range(ws):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(ws),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_two_gloo_ranks_reduce_time_and_work():
    pytest.importorskip("torch")
    outs = _run_ranks(CHILD)
    res = [json.loads(line[len("RESULT "):]) for o in outs for line in o.splitlines() if line.startswith("RESULT ")]
    assert sorted(r["rank"] for r in res) == [0, 1]
    for r in res:
        assert r["ws"] == 2
        assert r["max"] == 2.0          # the slowest rank sets the step time
        assert r["sum"] == 30.0         # work of all replicas


def test_reference_arm_runs_on_rank_zero_only():
    pytest.importorskip("torch")
    outs = _run_ranks(
        "import os, sys; sys.path.insert(0, os.environ['ROOT']); sys.argv = ['bench.py', '--impl', 'reference', "
        "'--workload', 'plain', '--steps', '1', '--warmup', '3', '--ref-seconds', '0.2']; import bench; "
        "bench.main()")
    lines = [json.loads(line) for o in outs for line in o.splitlines() if line.startswith("{")]
    assert len(lines) == 1                       # one JSON line, from rank 0
    line = lines[0]
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
