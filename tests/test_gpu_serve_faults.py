"""Host-side failures of single served fits: each fails alone, and every other fit in the same
server finishes bit for bit as it does in a server without the failure.

  * a request with a non-finite start point is refused at submission (GOO_ERR_ARG);
  * a fit cancelled while it waits for admission, and one cancelled while it is active,
    end with status GOO_FIT_CANCELLED, releasing their slot and event memory;
  * a fit whose admission fails its allocation (the server's test hook) ends with status
    GOO_FIT_ALLOC_FAILED and the queue moves on;
  * the finished-ticket list reports every one of these fits exactly once.
No GPU fault is involved: the failures are made on the host between steps.
"""
import numpy as np
import pytest

import synth
from oracle import toys as otoys

pytestmark = pytest.mark.gpu

KIN = synth.DALITZ_MASSES
TOYS = [(1710700, 6000), (1710701, 900), (1710702, 15_000), (1710703, 3000), (1710704, 8000), (1710705, 2000)]


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def setup(goo):
    ctx = goo.Context(0)
    spec = synth.c3_spec(n_mc=100_000)
    mc = synth.round_to_f32(synth.dalitz_candidates(100_000, 1710013, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]), spec)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    env = otoys.envelope(spec, theta)
    start = theta.copy()
    free = np.array([not p[2] for p in spec["params"]])
    start[free] *= 0.96
    return ctx, spec, model, theta, env, start


def _run(server, tickets, max_rounds=5000, between=None, drained=None):
    for r in range(max_rounds):
        if between is not None:
            between(r)
        q, a, d = server.step()
        if drained is not None:
            # tickets drained after this step: each finished, and each drained once
            for t in server.finished(cap=2):
                assert server.result(t) is not None and t not in drained
                drained.append(t)
            assert len(drained) == d
        if q == 0 and a == 0:
            break
    return {t: server.result(t) for t in tickets}


def test_failures_stay_with_their_fit(goo, setup):
    ctx, spec, model, theta, env, start = setup
    # reference: the six toys alone in one server
    ref_server = goo.Server(model, theta, envelope=env)
    ref_t = [ref_server.submit(n, s, start) for s, n in TOYS]
    ref = _run(ref_server, ref_t)
    assert all(r[2]["status"] == 0 for r in ref.values()), [r[2] for r in ref.values()]

    # the same toys among failing requests; two fit slots, so that some wait in the queue
    server = goo.Server(model, theta, envelope=env, max_fits=2)
    bad = start.copy()
    bad[np.flatnonzero(np.array([not p[2] for p in spec["params"]]))[0]] = np.nan
    with pytest.raises(goo.GooError) as e:
        server.submit(5000, 1710710, bad)
    assert e.value.code == goo.GOO_ERR_ARG
    tickets = {}
    tickets[0] = server.submit(TOYS[0][1], TOYS[0][0], start)
    t_active_cancel = server.submit(12_000, 1710711, start)   # cancelled after it is admitted
    tickets[1] = server.submit(TOYS[1][1], TOYS[1][0], start)
    t_queued_cancel = server.submit(4000, 1710712, start)     # cancelled while it waits
    t_alloc_fail = server.submit(7000, 1710713, start)        # its allocation fails at admission
    for i in range(2, len(TOYS)):
        tickets[i] = server.submit(TOYS[i][1], TOYS[i][0], start)
    server.fail_allocation(t_alloc_fail)
    server.cancel(t_queued_cancel)
    state = {"cancelled": False}

    def between(r):
        # after two rounds the second fit is active: cancel it between steps
        if r == 2 and not state["cancelled"]:
            server.cancel(t_active_cancel)
            state["cancelled"] = True

    drained = []
    everyone = list(tickets.values()) + [t_active_cancel, t_queued_cancel, t_alloc_fail]
    res = _run(server, everyone, between=between, drained=drained)
    assert state["cancelled"]
    # the finished list holds every fit once, failed ones included, and is empty afterwards
    assert sorted(drained) == sorted(everyone) and server.finished() == []
    assert res[t_active_cancel][2]["status"] == goo.GOO_FIT_CANCELLED
    assert res[t_queued_cancel][2]["status"] == goo.GOO_FIT_CANCELLED
    assert res[t_alloc_fail][2]["status"] == goo.GOO_FIT_ALLOC_FAILED
    for r in (res[t_active_cancel], res[t_queued_cancel], res[t_alloc_fail]):
        assert np.array_equal(r[0], start) and np.all(r[1] == 0) and r[2]["nll"] == np.inf
    # every other fit: bit for bit the result it has without the failures
    for i, t in tickets.items():
        got, want = res[t], ref[ref_t[i]]
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), i
        assert got[2]["iterations"] == want[2]["iterations"] and got[2]["status"] == 0
    # the server's memory is all free again, and it cannot cancel a finished fit
    assert server.stats()["arena_used"] == 0
    with pytest.raises(goo.GooError) as e:
        server.cancel(tickets[0])
    assert e.value.code == goo.GOO_ERR_STATE
    with pytest.raises(goo.GooError) as e:
        server.cancel(123456789)
    assert e.value.code == goo.GOO_ERR_ARG
