"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own
channel seed, combined by the max of their times (no data collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    from paper_1510_08886_gb300 import replicas
    dist = replicas.init("gloo")
    assert replicas.env() == (ws, rank, rank)
    seconds = 1.0 + rank          # rank 1 is the slow one
    rate, slowest = replicas.aggregate_rate(1000.0, seconds, dist)
    seed = replicas.replica_seed(20151029, rank)
    # every rank sees the same aggregate
    out.put((rank, rate, slowest, seed))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_by_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slowest, seed in res:
        assert slowest == 2.0
        assert rate == 2 * 1000.0 / 2.0
        assert seed == 20151029 + rank


def test_single_rank_needs_no_process_group():
    from paper_1510_08886_gb300 import replicas
    assert replicas.init("gloo") is None or os.environ.get("WORLD_SIZE", "1") != "1"
    assert replicas.aggregate_rate(10.0, 2.0, None) == (5.0, 2.0)
