"""The N > 1 bench path on CPU: gloo ranks use bench.py's barrier and
max-over-ranks timing reduction, and its slice sharding: each rank takes a
contiguous share of the kept range and one host-side sum-reduce of the heads
(the path's one exchange step) gives the full head."""
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
    from paper_2111_03011_gb300.shard import reduce_heads, slice_share
    from tests.plan_emulator import emulate
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True)
    k = tn.tn_plan_get_stats(plan)["n_sliced"]
    b, e = slice_share(0, 1 << k, rank, world)          # the bench's split of the kept range
    H = emulate(tn.tn_plan_describe(plan, with_data=True), cfg["tails"], cfg["open_qubits"], range(b, e))
    t = torch.from_numpy(np.ascontiguousarray(H))
    reduce_heads(t)                                     # the bench's exchange step
    dist.destroy_process_group()
    q.put((rank, (b, e, t.numpy())))


@pytest.mark.parametrize("world", [2, 3])
def test_slice_ranges_shard_across_ranks_and_sum(world):
    """Slices are independent: gloo ranks take contiguous shares of the slice
    range (bench.py's split, ragged at 3 ranks of 16 slices), and the sum of
    their heads (bench.py's host-side reduce) equals the oracle's full sum on
    every rank."""
    import multiprocessing as mp

    import numpy as np

    import circuit_inputs as ci
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = sorted(res[r][:2] for r in range(world))
    assert shares[0][0] == 0 and shares[-1][1] == 16
    assert all(a[1] == b[0] for a, b in zip(shares, shares[1:]))        # contiguous, disjoint, covering
    assert max(e - b for b, e in shares) - min(e - b for b, e in shares) <= 1
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    se = [(g, l) for (g, l, k, v) in cfg["edges"]]
    ref = O.sparse_state_from_vector(O.sliced_statevector(cfg["circuit"], se), cfg["open_qubits"], cfg["tails"])
    for r in range(world):
        assert np.abs(res[r][2] - ref).max() < 1e-12


def test_slice_share_tiles_any_range():
    from paper_2111_03011_gb300.shard import slice_share
    for (b, e) in [(0, 64), (3, 10), (5, 5), (0, 1)]:
        for world in (1, 2, 3, 4, 8, 100):
            parts = [slice_share(b, e, r, world) for r in range(world)]
            assert parts[0][0] == b and parts[-1][1] == e
            assert all(p[1] == q[0] for p, q in zip(parts, parts[1:]))
            assert max(p[1] - p[0] for p in parts) - min(p[1] - p[0] for p in parts) <= 1
    with pytest.raises(ValueError):
        slice_share(0, 4, 2, 2)
