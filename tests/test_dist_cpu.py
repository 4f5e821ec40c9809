"""The N > 1 bench path on CPU: world-size-2 gloo ranks use bench.py's barrier
and max-over-ranks timing reduction (the path runs independent replicas, so
timing is the only cross-rank exchange)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    bench._barrier(ws)
    m = bench._max(ws, 10.0 + rank)
    bench._barrier(ws)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, m))


def test_two_rank_barrier_and_max_over_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 11.0, 1: 11.0}


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch
    import torch.distributed as dist

    import circuit_inputs as ci
    import paper_2111_03011_gb300 as tn
    from tests.plan_emulator import emulate
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True)
    k = tn.tn_plan_get_stats(plan)["n_sliced"]
    per = (1 << k) // world
    H = emulate(tn.tn_plan_describe(plan, with_data=True), cfg["tails"], cfg["open_qubits"],
                range(rank * per, (rank + 1) * per))
    t = torch.from_numpy(np.ascontiguousarray(H))
    dist.all_reduce(t)                       # the heads of the slice shards add up
    dist.destroy_process_group()
    q.put((rank, t.numpy()))


def test_slice_ranges_shard_across_ranks_and_sum():
    """Slices are independent: two gloo ranks take half of the slice range each
    and the sum of their heads (one all-reduce) equals the oracle's full sum."""
    import multiprocessing as mp

    import numpy as np

    import circuit_inputs as ci
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    se = [(g, l) for (g, l, k, v) in cfg["edges"]]
    ref = O.sparse_state_from_vector(O.sliced_statevector(cfg["circuit"], se), cfg["open_qubits"], cfg["tails"])
    for r in (0, 1):
        assert np.abs(res[r] - ref).max() < 1e-12
