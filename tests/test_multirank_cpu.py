"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks (the GPU path runs
independent replicas; its only cross-rank steps are the barrier and the maximum
of the timed region), and the reference arm under torchrun (rank 0 alone runs
and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, rank, world)
    ms = 10.0 + 5.0 * rank                      # the ranks disagree; the job takes the slowest
    got = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, bench.whole_job_rate(1000, world, 4, got)))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, got, rate in res:
        assert got == 15.0
        assert rate == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_reference_arm_under_torchrun_prints_once():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_bench_lat_metrics_follow_their_definition():
    """bench.py's LAT-vs-synchronised figures (Sec. 7.4) against the same
    definitions written independently in the oracle's LAT tests, on seeded data
    with a dense region, floor-level cells and a sign pattern in the differences."""
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import bench
    from test_oracle_lat import lat_metrics
    rng = np.random.default_rng(8)
    sync = 10 ** rng.uniform(-10, 0, 5000)
    lat = sync * (1 + 1e-3 * rng.normal(size=5000))
    lat[:50] = 1e-9 * rng.uniform(0.5, 2.0, 50)   # cells crossing the dense threshold
    got = bench.lat_vs_sync_metrics(torch, torch.from_numpy(lat), torch.from_numpy(sync), 1e-11)
    want = lat_metrics(lat, sync, 1e-11)
    for k, w in zip(("L1", "L2", "Linf", "C_logrho", "J_dense"), want):
        assert got[k] == pytest.approx(float(w), rel=1e-12), k
    assert got["J_dense"] < 1.0
