"""Event sharding over ranks (one process per GPU) and the deterministic combine.

Events are independent (the paper's MPI scheme divides the dataset among processes, Sec. 4):
rank r of N evaluates the contiguous event range shard_range(n, r, N) with
goo_nll_partial, one all-gather gives every rank every shard's record, and the records are
added in rank order with compensated arithmetic (goo_combine_partials).  Every rank
therefore obtains the same bits whatever order the collective uses internally.

torch.distributed carries the records (NCCL between GPUs, gloo on the host); the
arithmetic is the library's.
"""
import numpy as np

from . import goo


def shard_range(n, rank, world):
    """[begin, end) of rank's contiguous share of n events (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    q, r = divmod(int(n), int(world))
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def allgather_records(record, group=None, device=None):
    """All ranks' records (rows in rank order) from this rank's record."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.as_tensor(np.asarray(record, dtype=np.float64), device=device)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return np.stack([o.cpu().numpy() for o in out])


def combine(records, n_params):
    """(nll, grad, events) of records added in row order with compensation."""
    tot = goo.combine_partials(records, n_params)
    return tot[0] + tot[1], tot[3:].copy(), int(round(tot[2]))


def nll_grad_sharded(model, ds, theta, precision, rank, world, group=None, device=None, want_grad=True):
    """NLL and gradient of the whole dataset, ds holding all events or this rank's shard.

    When ds holds n_total events on every rank, pass the full dataset: each rank evaluates
    only shard_range(n_total, rank, world).  Returns the same (nll, grad) on every rank.
    """
    b, e = shard_range(ds.n, rank, world)
    rec = model.nll_partial(ds, b, e, theta, precision, want_grad=want_grad)
    recs = allgather_records(rec, group=group, device=device)
    nll, grad, _ = combine(recs, model.n_params)
    return nll, grad
