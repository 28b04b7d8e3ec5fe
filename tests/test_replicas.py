"""Multi-GPU layout on the host: the bench's replica plumbing (one process per GPU,
independent right-hand sides per rank, timing collectives only) run as two `gloo`
ranks on CPU. Checks the per-rank seed shift (rank 0 = the single-GPU workload, no
seed shared across ranks), the max over ranks of a timed region, the sum of units
and the whole-job rate = all units / the slowest rank's time, and that world size 1
needs no process group."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rep = bench.Replicas("gloo")
w = bench.workload("cube_th_p3_64")
seeds = rep.seeds(w["seeds"], 24)
rep.barrier()
out = dict(rank=rep.rank, world=rep.world, seeds=seeds, parallelism=rep.parallelism,
           ms=rep.max(10.0 + 5.0 * rep.rank), units=rep.sum(3 * (rep.rank + 1)),
           rate=rep.job_rate(4 * (rep.rank + 1), 1.0 + rep.rank),
           vec_max=rep.reduce([rep.rank, -rep.rank, 2.5], "max"),
           vec_sum=rep.reduce([rep.rank, 0.25], "sum"))
every = [None] * rep.world
dist.all_gather_object(every, seeds)
out["all_seeds"] = every
rep.close()
print("RESULT " + json.dumps(out), flush=True)
"""


DEPARTING = r"""
import sys, time
sys.path.insert(0, sys.argv[1])
import bench
rep = bench.Replicas("gloo", timeout_s=20)
rep.barrier()
if rep.rank == 1:
    sys.exit(0)                     # leaves between steps, with no collective in flight
t0 = time.time()
try:
    rep.max(1.0)
    print("RESULT joined", flush=True)
except Exception as e:
    print("RESULT raised %.1f %s" % (time.time() - t0, type(e).__name__), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(world, script):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", script, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    texts = []
    try:
        for p in procs:
            text, _ = p.communicate(timeout=240)
            texts.append((p.returncode, text))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
                p.wait()
    return texts


def _run_ranks(world):
    outs = []
    for rc, text in _launch(world, WORKER):
        assert rc == 0, text
        line = [ln for ln in text.splitlines() if ln.startswith("RESULT ")]
        assert line, text
        outs.append(json.loads(line[-1][len("RESULT "):]))
    return sorted(outs, key=lambda o: o["rank"])


def test_two_gloo_ranks():
    import bench
    o0, o1 = _run_ranks(2)
    base = bench.workload("cube_th_p3_64")["seeds"]
    # rank 0 solves exactly the single-GPU workload; rank 1 the same list shifted by the stride
    assert o0["seeds"] == [base[j % len(base)] for j in range(24)]
    assert o1["seeds"] == [s + bench.Replicas.SEED_STRIDE for s in o0["seeds"]]
    assert not set(o0["seeds"]) & set(o1["seeds"])
    for o in (o0, o1):
        assert o["world"] == 2 and o["parallelism"] == "replicas x2"
        assert o["all_seeds"] == [o0["seeds"], o1["seeds"]]
        assert o["ms"] == 15.0                       # the slowest rank's time
        assert o["units"] == 3.0 + 6.0               # units summed over ranks
        assert o["rate"] == pytest.approx((4 + 8) / 2.0)
        assert o["vec_max"] == [1.0, 0.0, 2.5]
        assert o["vec_sum"] == [1.0, 0.5]


def test_single_rank_needs_no_process_group():
    import torch.distributed as dist

    import bench
    rep = bench.Replicas("gloo", env={})
    assert (rep.world, rep.rank, rep.local) == (1, 0, 0)
    assert not dist.is_initialized()
    assert rep.parallelism == "1 GPU"
    assert rep.seeds([5, 6], 3) == [5, 6, 5]
    assert rep.max(2.5) == 2.5 and rep.sum(4) == 4.0 and rep.job_rate(10, 2.0) == 5.0
    rep.barrier()
    rep.close()


def test_departed_rank_ends_the_next_collective_with_an_error():
    """Failure detection on the host: rank 1 leaves between steps; rank 0's next
    timing collective fails with an error (the peer's closed connection, at the latest
    the process group's 20 s timeout) instead of waiting forever."""
    (rc0, t0), (rc1, t1) = _launch(2, DEPARTING)
    assert rc1 == 0, t1
    line = [ln for ln in t0.splitlines() if ln.startswith("RESULT ")]
    assert line and line[-1].startswith("RESULT raised"), t0
    assert float(line[-1].split()[2]) <= 30.0
