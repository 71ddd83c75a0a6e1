"""The N > 1 host path of the benchmark on CPU (gloo, world size 2): the
self-join does not shard into a collective -- N GPUs run N independent
replicas -- so what is shared is the rendezvous, the barrier and the
max-over-ranks timing, and the reference arm's rank-0-only rule."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    t = bench.max_over_ranks(10.0 + 5.0 * r, w)            # per-rank step time, ms
    v = bench.replica_value(w, cells=1000, steps=2, total_ms=t)
    q.put((r, w, t, v))
    dist.destroy_process_group()


def test_gloo_rendezvous_barrier_and_max_over_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for r, w, t, v in got:
        assert w == 2 and t == 15.0                          # the slowest rank's time
        assert v == pytest.approx(2 * 1000 * 2 / 15e-3 / 1e9)  # all replicas' cells / max time


def test_reference_arm_prints_one_line_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--series-length", "4096", "--window", "64", "--steps", "1",
           "--warmup", "3",
           "--ref-step-s", "0.3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
