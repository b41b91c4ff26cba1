"""bench.py's multi-GPU form is replicas only: each rank runs independent
problems, timing is bracketed by barriers and the whole-job rate is all ranks'
pixel-iterations over the slowest rank's time. The reduction helpers are
checked here with world_size-2 gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    bench.rank_barrier(ws)
    # rank r processed (r + 1) * 1e6 pixel-iterations in (r + 1) * 0.5 s
    rate, slow = bench.replica_rate((rank + 1) * 1e6, (rank + 1) * 0.5, ws, device="cpu")
    mx = bench.rank_max(float(rank), ws, device="cpu")
    q.put((rank, rate, slow, mx))
    dist.destroy_process_group()


def test_replica_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, rate, slow, mx in out:
        assert slow == pytest.approx(1.0)          # the slowest rank's time
        assert rate == pytest.approx(3.0)          # (1 + 2) Mpixel-iters / 1 s
        assert mx == 1.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    rate, slow = bench.replica_rate(2e6, 0.5, 1)
    assert (rate, slow) == (4.0, 0.5)
    assert bench.rank_max(7.0, 1) == 7.0
