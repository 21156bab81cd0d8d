"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2).

The method shards as independent replicas (one lattice per GPU, no data-path
collective); the only cross-rank operations are the barrier and the maximum
of the per-rank times.  Here those run as two gloo processes on the host.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [1.5, 2.5][rank]                 # the second replica is the slow one
    m = bench.max_over_ranks(secs, world, "cpu")
    dist.barrier()
    q.put((rank, m, bench.job_mlups(1000, 10, world, m)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, val in out:
        assert m == 2.5
        assert val == pytest.approx(1000 * 10 * 2 / 2.5 / 1e6)


def test_reference_arm_two_ranks_prints_one_line():
    """bench.py --impl reference under torchrun with two ranks: rank 0 alone
    times the oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
                        "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["warmup"] >= 3
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["higher_is_better"] is True
