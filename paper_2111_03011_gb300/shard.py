"""Slice ranges sharded over several GPUs, one process per GPU.

Slices are independent sub-tasks whose contributions add up (Results: the
2^16 sub-tasks of the 53-qubit run went to 512 GPUs; Supplement, slicing:
the head is the sum over the kept slices).  A kept range [begin, end) is cut
into contiguous per-rank ranges; every rank contracts its range into its own
head on its own GPU, and one exchange step sums the heads: a sum-reduce of
the L x 2^h complex128 head (1 MiB for 64 x 1024), done on the host over a
torch.distributed process group (gloo), since each GPU machine holds one GPU.
Rank 0 then owns the summed head and its fidelity estimate, the fraction of
all slices the ranks accumulated.
"""
from __future__ import annotations


def slice_share(begin: int, end: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous part of [begin, end) for `rank` of `world`: sizes differ by
    at most one slice, ranks in order, the parts tile the range exactly."""
    if world < 1 or not 0 <= rank < world or end < begin:
        raise ValueError("bad shard arguments")
    n = end - begin
    return begin + (rank * n) // world, begin + ((rank + 1) * n) // world


def reduce_heads(head_host, group=None):
    """Sum a CPU complex128 head over all ranks of `group`, in place."""
    import torch
    import torch.distributed as dist
    assert head_host.dtype == torch.complex128 and head_host.device.type == "cpu"
    dist.all_reduce(torch.view_as_real(head_host), op=dist.ReduceOp.SUM, group=group)
    return head_host
