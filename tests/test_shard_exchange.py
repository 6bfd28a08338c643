"""The exchange step of the feature-sharded iteration, on CPU: gloo ranks on 127.0.0.1.

One problem split by columns needs, per MM iteration, every shard's partial
sums (per-edge ||b||^2 pieces and the scalar pieces of d_m and the stopping
rule) on every shard, in shard order, so that each shard's reduction adds them
in the same order and all shards keep the same state.  These tests run the
binding's exchange helpers in real processes: the gathered rows arrive in rank
order on every rank, and an ordered sum of values whose floating-point sum
depends on the order gives the rank-order result everywhere.
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
import torch
import torch.distributed as dist
dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
from paper_1409_2065_gb300 import binding as B
part = torch.arange(6, dtype=torch.float64) + 100.0 * rank
allp = B.allgather_parts(part)
vals = [1e16, -1e16, 1.0][:ws]
s = B.ordered_sum([vals[rank], 2.0 * rank])
out = {"rank": rank, "ws": ws, "rows": allp.tolist(), "sum": s.tolist()}
dist.barrier()
dist.destroy_process_group()
print("RESULT " + json.dumps(out), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(ws, timeout=180):
    port = _free_port()
    procs = []
    for r in range(ws):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(ws),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    res = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        res += [json.loads(ln[len("RESULT "):]) for ln in o.splitlines() if ln.startswith("RESULT ")]
    return sorted(res, key=lambda r: r["rank"])


@pytest.mark.parametrize("ws", [2, 3])
def test_allgather_in_rank_order_and_ordered_sum(ws):
    pytest.importorskip("torch")
    res = _run(ws)
    assert [r["rank"] for r in res] == list(range(ws))
    expect_rows = [[k + 100.0 * q for k in range(6)] for q in range(ws)]
    for r in res:
        assert r["ws"] == ws
        assert r["rows"] == expect_rows              # every rank sees every shard, in shard order
        assert r["sum"] == res[0]["sum"]             # bit-identical on every rank
    # (1e16 + -1e16) + 1 = 1 in rank order, while 1e16 + (-1e16 + 1) would give 0
    assert res[0]["sum"][0] == (1.0 if ws == 3 else 0.0)
    assert res[0]["sum"][1] == float(sum(2.0 * q for q in range(ws)))
