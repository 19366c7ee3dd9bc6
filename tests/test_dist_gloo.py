"""The sharded NLL protocol on two gloo ranks (CPU): contiguous shard ranges, an all-gather
of the per-shard records and the library's ordered, compensated combine reproduce the
oracle's NLL and gradient of the whole dataset, identically on every rank (Sec. 4: the
dataset is divided among processes)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synth
        from oracle import model as om
        from paper_1710_08826_gb300 import dist as gd
        spec = synth.c1_spec()
        cols = synth.gen_c1(n=n, seed=31)
        theta = np.array(synth.param_values(spec)) * 1.02
        b, e = gd.shard_range(n, rank, world)
        nll, g = om.TreeModel(spec).nll_grad({k: v[b:e] for k, v in cols.items()}, theta)
        rec = np.concatenate([[nll, 0.0, float(e - b)], g])
        recs = gd.allgather_records(rec)
        tot, grad, events = gd.combine(recs, len(theta))
        q.put((rank, tot, grad.tolist(), events))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_partition():
    from paper_1710_08826_gb300.dist import shard_range
    for n in (0, 1, 7, 1000, 100_003):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def test_two_gloo_ranks_match_the_full_oracle():
    import torch.multiprocessing as mp
    from paper_1710_08826_gb300 import buildlib
    buildlib.build()  # the combiner is the library's (host code; no GPU needed)
    import synth
    from oracle import model as om
    n, world = 20_001, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = synth.c1_spec()
    theta = np.array(synth.param_values(spec)) * 1.02
    rnll, rg = om.TreeModel(spec).nll_grad(synth.gen_c1(n=n, seed=31), theta)
    (_, nll0, g0, ev0), (_, nll1, g1, ev1) = out
    assert nll0 == nll1 and g0 == g1 and ev0 == ev1 == n   # identical bits on both ranks
    assert abs(nll0 - rnll) <= 1e-12 * abs(rnll)
    np.testing.assert_allclose(g0, rg, rtol=1e-10, atol=1e-10 * np.abs(rg).max())


class _HostServer:
    """A stand-in with goo.Server's submit / step / result protocol that "fits" each request
    on the host (the oracle's C1 NLL and gradient on a seeded sample of the request's size),
    one request per step, so that the split and gather logic runs without a GPU."""

    def __init__(self):
        self.queue, self.done, self.next = [], {}, 1

    def submit(self, n, seed, theta_start):
        t = self.next
        self.next += 1
        self.queue.append((t, n, seed, np.asarray(theta_start, dtype=np.float64)))
        return t

    def step(self):
        import synth
        from oracle import model as om
        if self.queue:
            t, n, seed, th = self.queue.pop(0)
            spec = synth.c1_spec()
            nll, g = om.TreeModel(spec).nll_grad(synth.gen_c1(n=n, seed=seed), th)
            self.done[t] = (th - 1e-6 * g, np.abs(g), {"status": 0, "nll": nll})
        return len(self.queue), 0, len(self.done)

    def result(self, t):
        return self.done[t]


def _requests():
    import synth
    theta = np.array(synth.param_values(synth.c1_spec()))
    sizes = [5000, 300, 12_000, 800, 800, 7000, 2500, 40, 9000]
    return [(n, 1710900 + i, theta * (1 + 0.01 * i)) for i, n in enumerate(sizes)]


def _serve_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1710_08826_gb300 import dist as gd
        table = gd.serve_fits(_HostServer, _requests(), rank, world)
        q.put((rank, table.tolist()))
    finally:
        dist.destroy_process_group()


def test_split_fits_balances_whole_fits():
    from paper_1710_08826_gb300.dist import split_fits
    sizes = [5000, 300, 12_000, 800, 800, 7000, 2500, 40, 9000]
    for world in (1, 2, 3, 4, 16):
        shares = split_fits(sizes, world)
        assert sorted(i for s in shares for i in s) == list(range(len(sizes)))   # each fit once
        loads = [sum(sizes[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(sizes)                            # greedy bound
        assert shares == split_fits(sizes, world)                               # deterministic
    assert split_fits(sizes, 2) == [[0, 2, 3, 4, 7], [1, 5, 6, 8]]   # loads 18,640 and 18,800 events


def test_two_gloo_ranks_serve_whole_fits_like_one():
    import torch.multiprocessing as mp
    from paper_1710_08826_gb300 import dist as gd
    reqs = _requests()
    single = np.array(gd.serve_share(_HostServer(), reqs, list(range(len(reqs)))))
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serve_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    t0, t1 = np.array(out[0][1]), np.array(out[1][1])
    assert np.array_equal(t0, t1)          # every rank holds the whole table
    assert np.array_equal(t0, single)      # and it equals the single-rank run, row for row
