"""The multi-rank bench path on CPU (gloo, world size 2).

`bench.py --gpus N` runs one independent replica per rank (each its own scan,
no data-path collective) and reports the whole job: units summed over ranks,
time = the slowest rank.  These tests run that aggregation across two gloo
processes; no GPU is involved.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, units, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(times[rank], units[rank], dist)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, u))


def _run(times, units):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, units, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_aggregate_sums_units_and_takes_the_slowest_rank():
    res = _run([1.25, 2.5], [10_385_229, 10_400_001])
    for _, t, u in res:
        assert t == 2.5                       # max over ranks
        assert u == 10_385_229 + 10_400_001   # whole-job units
    # every rank reports the same whole-job numbers
    assert res[0][1:] == res[1][1:]


def test_aggregate_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.0, 7, None) == (3.0, 7)


def test_reference_arm_under_torchrun_prints_one_line(orc):
    """`bench.py --impl reference` launched as two ranks (the driver's N > 1
    launch): rank 0 times the oracle and prints the one JSON line, the other
    rank exits 0 without work."""
    import json
    import subprocess
    import sys
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "room"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
