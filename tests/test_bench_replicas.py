"""The multi-GPU form of the benchmark is replicas only: every rank solves its
own copy of the workload, the job's time is the slowest rank's, and the value
counts the units of all ranks.  These host-side pieces run here as two gloo
ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import io, contextlib, json, os, sys
sys.path.insert(0, os.environ["TS_ROOT"])
import bench
dist, rank, ws = bench._dist("gloo")
assert ws == 2 and rank == int(os.environ["RANK"])
t = bench._max_over_ranks(dist, 1.0 + rank)
assert t == 2.0, t
rate = bench._job_rate(ws, 1000, 7, 31, t)
assert abs(rate - 2 * 1000 * 7 * 31 / 2.0) < 1e-9
# the reference arm prints its one line on rank 0 only
if rank == 1:
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(None)
    assert buf.getvalue() == ""
dist.barrier()
dist.destroy_process_group()
print("rank", rank, "ok", flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_job_rate():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), TS_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        try:
            out, _ = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            p.kill()
            out, _ = p.communicate()
        outs.append(out)
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"rank {rank} ok" in out, out
