"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own
channel seed, combined by the max of their times (no data collective).
The solver work of a rank runs on the fp64 oracle here (no GPU): each rank
advances its own replica, and its result must be the one the same seed
gives in a single process -- the ranks share nothing but the timing."""
import os
import socket

import numpy as np
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


REPLICA = ("D2V16", 3, 1, 16, 0.1)      # velocity set, order, Nx, Ny, Kn
STEPS = 40


def _replica_mdot(rank):
    import oracle
    from lbm_inputs import DVM_TABLES, rho_field
    from oracle import dvm
    from paper_1510_08886_gb300 import replicas
    name, N, Nx, Ny, Kn = REPLICA
    e, w, c = dvm.dvm2d(name, DVM_TABLES)
    ch = oracle.Channel(e, w, c, N, Nx, Ny, Kn, oracle.force_for_mach(Kn, 1e-2))
    ch.init(rho_field(Nx, Ny, seed=replicas.replica_seed(20151029, rank), amplitude=1e-2))
    ch.step(STEPS)
    return ch.mass_flow(), float(np.sum(ch.f))


def _solver_worker(rank, ws, port, out):
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    from paper_1510_08886_gb300 import replicas
    dist = replicas.init("gloo")
    dist.barrier()
    t0 = time.perf_counter()
    mdot, mass = _replica_mdot(rank)
    dt = time.perf_counter() - t0
    Nx, Ny = REPLICA[2], REPLICA[3]
    rate, slowest = replicas.aggregate_rate(Nx * Ny * STEPS, dt, dist)
    out.put((rank, mdot, mass, rate, slowest, dt))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_run_their_own_replica():
    """Each rank advances its own seeded channel with no exchange of solver
    data; the whole-job rate is all ranks' node updates over the slowest
    rank's time, and each rank's mass flow and mass are bitwise those of a
    single-process run of its seed."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_solver_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    Nx, Ny = REPLICA[2], REPLICA[3]
    slowest = max(r[5] for r in res)
    for rank, mdot, mass, rate, sl, dt in res:
        assert sl == slowest
        assert rate == pytest.approx(2 * Nx * Ny * STEPS / slowest, rel=1e-12)
        ref_mdot, ref_mass = _replica_mdot(rank)
        assert mdot == ref_mdot and mass == ref_mass
    # the replicas are different channels (different seeds)
    assert res[0][1] != res[1][1]
