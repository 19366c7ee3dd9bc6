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


# ---------------------------------------------------------------------------------------
# served toy fits: whole fits per rank (independent replicas of the server)
# ---------------------------------------------------------------------------------------
def split_fits(sizes, world):
    """Whole fits per rank: each request, in descending order of its event count (ties: lower
    index first), goes to the rank with the fewest events so far (ties: lower rank).  Returns
    world lists of request indices, each in ascending order.  Deterministic, so every rank
    computes the same split without communicating."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError(f"world {world}")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    share = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        share[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(s) for s in share]


def serve_share(server, requests, indices):
    """Runs requests[i] = (n_events, seed, theta_start) for i in indices through one server
    (submitted in index order, stepped until the server is idle) and returns, per index, the
    row [index, status, nll, theta..., errors...]."""
    tickets = {i: server.submit(*requests[i]) for i in indices}
    while True:
        q, a, _ = server.step()
        if q == 0 and a == 0:
            break
    rows = []
    for i in indices:
        th, err, info = server.result(tickets[i])
        rows.append(np.concatenate([[float(i), float(info["status"]), float(info["nll"])], th, err]))
    return rows


def serve_fits(make_server, requests, rank, world, group=None, device=None):
    """The served study over ranks: rank r runs its share split_fits(...)[r] through its own
    server (make_server() on this rank's GPU), then one all-gather gives every rank every
    fit's row; returns the rows in request order (an array [len(requests), 3 + 2 P])."""
    import torch
    import torch.distributed as dist
    shares = split_fits([r[0] for r in requests], world)
    mine = serve_share(make_server(), requests, shares[rank]) if shares[rank] else []
    P = len(requests[0][2])
    width = 3 + 2 * P
    most = max(len(s) for s in shares)
    buf = np.full((most, width), np.nan)
    for k, row in enumerate(mine):
        buf[k] = row
    t = torch.as_tensor(buf, device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    table = np.full((len(requests), width), np.nan)
    for r, o in enumerate(out):
        rows = o.cpu().numpy()
        for k, i in enumerate(shares[r]):
            table[i] = rows[k]
    return table
