"""Multi-GPU runs are independent replicas (the method has no exchange step): each
rank evolves its own batch with its own seeds, and bench.py only needs a barrier
and a max over ranks of the timed interval.  That host logic, on two gloo ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2307_07999_gb300 import workloads as W

    got_ws, got_rank, local = bench.dist_setup()
    assert (got_ws, got_rank, local) == (ws, rank, rank)
    bench.barrier(ws)
    # the slowest rank's interval is the job's
    t = bench.max_over_ranks(10.0 + rank, ws)
    evs, pps = W.batched_uneven(rank=rank)
    seeds = [e.seed for e in evs] + [p.seed for p in pps]
    out[rank] = (t, seeds)
    bench.barrier(ws)
    dist.destroy_process_group()


def test_two_gloo_replicas_barrier_max_and_distinct_seeds():
    ws = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0
    s0, s1 = set(res[0][1]), set(res[1][1])
    assert len(s0) == len(res[0][1]) and not (s0 & s1)  # every event of every replica is its own


def _pool_rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2307_07999_gb300 import api

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    rng = np.random.default_rng(rank)
    tau = np.linspace(0.1, 1.0, 7)
    cnt = np.full(7, 1000.0 * (rank + 1))
    cnt[0] = 0.0  # a row without particles on every rank stays zero
    tab = np.column_stack([tau, rng.random((7, 3)), cnt])
    tab[0, 1:4] = 0.0
    out[rank] = (tab, api.pool_broadening(tab))
    bad = np.column_stack([tau + rank, rng.random((7, 3)), cnt])
    try:
        api.pool_broadening(bad)
        out[f"err{rank}"] = False
    except ValueError:
        out[f"err{rank}"] = True
    dist.destroy_process_group()


def test_pool_broadening_is_the_count_weighted_mean_over_replicas():
    import numpy as np

    ws = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_pool_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    (t0, p0), (t1, p1) = res[0], res[1]
    want = t0.copy()
    want[:, 4] = t0[:, 4] + t1[:, 4]
    want[1:, 1:4] = (t0[1:, 1:4] * t0[1:, 4:5] + t1[1:, 1:4] * t1[1:, 4:5]) / want[1:, 4:5]
    assert np.allclose(p0, want, rtol=1e-15, atol=0) and np.array_equal(p0, p1)
    assert np.all(p0[0, 1:4] == 0)
    assert res["err0"] and res["err1"]
