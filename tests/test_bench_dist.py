"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

Plans are independent, so N GPUs run N replicas with no collective on the data
path; the only cross-rank steps are the barrier around the timed region, the
maximum of the step time, and the whole-job sums.  These run here as two gloo
ranks.  The reference arm under torch.distributed.run must print one JSON line
from rank 0 and let the other rank exit 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "VMAT_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_setup(world)
    bench.barrier(w)
    res = {"rank": r, "world": w, "local": local,
           "max": bench.max_over_ranks(rank + 1.0, w),
           "sum": bench.sum_over_ranks(rank + 1.0, w),
           # rank r moved (r + 1) GB in 0.5 (r + 1) s: 3 GB in 1 s for the job
           "gbs": bench.whole_job_gbs((rank + 1) * 1e9, 0.5 * (rank + 1), w)}
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put(res)


def test_collectives_and_whole_job_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1] and all(d["world"] == 2 for d in res)
    assert all(d["max"] == 2.0 and d["sum"] == 3.0 for d in res)
    assert all(abs(d["gbs"] - 3.0) < 1e-12 for d in res)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0 and bench.sum_over_ranks(4.0, 1) == 4.0
    assert bench.whole_job_gbs(2e9, 0.5, 1) == 4.0


def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, VMAT_BENCH_BACKEND="gloo", PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
