"""Serving with continuous batching: runs submitted while others are on the
GPU are admitted as slots and memory free up, and every result (MCS reached,
extinction flag, counts, lattice) is bit-identical to running it alone."""
import numpy as np
import pytest

import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300 import workloads as W
from paper_2508_16639_gb300.build import build
from paper_2508_16639_gb300.serve import request_spec, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _reqs(n, seed, L_range=(50, 300), budget=(20, 200)):
    return W.request_stream(n=n, seed=seed, rate_per_s=200.0, L_range=L_range, budget_range=budget)


def _alone(sp):
    g = E.Lattice(sp["L"], sp["S"], sp["digraph"], sp["rates"], sp["seed"], p_empty=sp["p_empty"],
                  log_every=10, stop_at_extinction=sp["stop_at_extinction"])
    g.run(sp["max_mcs"])
    ms, log = g.counts_log()
    return g.mcs, g.snapshot(), log[-1]


@pytest.mark.parametrize("arena_mb,max_slots", [(256, 64), (1, 8)])
def test_served_runs_match_single_runs(arena_mb, max_slots):
    reqs = _reqs(24, seed=5)
    srv = E.Server(arena_bytes=arena_mb << 20, max_slots=max_slots, keep_lattice=True,
                   chunks_per_step=2)
    ids = {}
    queued_seen = 0
    # arrivals interleaved with steps: 6 submissions, a step, 6 more, ...
    for k in range(0, len(reqs), 6):
        for r in reqs[k:k + 6]:
            ids[srv.submit(request_spec(r))] = r
        srv.step()
        queued_seen = max(queued_seen, srv.stats()[1])
    done = set()
    for _ in range(10000):
        done.update(srv.poll())
        if len(done) == len(reqs):
            break
        srv.step()
    assert len(done) == len(reqs)
    if arena_mb == 1:
        assert queued_seen > 0   # memory admission made runs wait
    for rid, r in ids.items():
        sp = request_spec(r)
        mcs, ext, cnt, lat = srv.result(rid, lattice=True)
        m1, lat1, c1 = _alone(sp)
        assert mcs == m1, rid
        assert np.array_equal(lat, lat1), rid
        assert np.array_equal(cnt[:sp["S"] + 1], c1), rid
        assert ext == (sp["stop_at_extinction"] and (c1[1:] > 0).sum() <= 1)
    assert srv.stats() == (0, 0, 0)


def test_served_runs_match_the_replay_oracle():
    """A served mix -- small runs and three at L = 1000 .. 1600 from the top of
    the serving workload's range -- against the schedule-v1 replay oracle run
    by itself: MCS reached (stasis or budget), counts and lattice."""
    import oracle as O
    small = _reqs(10, seed=21, L_range=(50, 300), budget=(20, 120))
    big = _reqs(3, seed=22, L_range=(1000, 1600), budget=(20, 30))
    reqs = small[:5] + big + small[5:]
    srv = E.Server(arena_bytes=256 << 20, max_slots=16, keep_lattice=True, chunks_per_step=2)
    ids = {}
    for k in range(0, len(reqs), 4):
        for r in reqs[k:k + 4]:
            ids[srv.submit(request_spec(r))] = r
        srv.step()
    done = set()
    for _ in range(10000):
        done.update(srv.poll())
        if len(done) == len(reqs):
            break
        srv.step()
    assert len(done) == len(reqs)
    assert max(r["L"] for r in reqs) >= 1000
    for rid, r in ids.items():
        sp = request_spec(r)
        D = O.circulant(sp["S"], r["K"])
        I, P, X = sp["rates"]
        lat, log, mend = O.run_observed(O.init(sp["L"], sp["S"], sp["p_empty"], sp["seed"]), D, I, P, X,
                                        sp["seed"], sp["max_mcs"], log_every=10,
                                        stop_at_extinction=sp["stop_at_extinction"])
        mcs, ext, cnt, glat = srv.result(rid, lattice=True)
        assert mcs == mend, rid
        assert np.array_equal(glat, lat), rid
        assert np.array_equal(cnt[:sp["S"] + 1], log[-1]), rid


def test_serve_loop_reports_latency():
    reqs = _reqs(40, seed=9, L_range=(50, 200), budget=(20, 100))
    out = serve(reqs, time_scale=0.05, arena_bytes=64 << 20, max_slots=32, chunks_per_step=2)
    assert out["runs"] == 40 and out["runs_per_s"] > 0
    assert 0 < out["p50_latency_s"] <= out["p99_latency_s"]
    b = out["latency_breakdown"]
    assert 0 <= b["queue_p50_s"] <= b["queue_p99_s"] and 0 < b["service_p50_s"] <= b["service_p99_s"]
    assert b["service_p99_s"] <= out["p99_latency_s"] + 1e-6


def test_submit_rejects_runs_larger_than_the_arena():
    srv = E.Server(arena_bytes=64 << 10, max_slots=4)
    r = _reqs(1, seed=1, L_range=(600, 601))[0]
    with pytest.raises(E.EscgError):
        srv.submit(request_spec(r))


def test_cancel_queued_and_running_runs():
    """A queued run cancelled before admission reports MCS 0; a running run
    cancelled between steps stops at the MCS it reached, with the lattice a
    run alone reaches at that MCS; the other runs are unaffected and the
    slot and arena memory are reused."""
    reqs = _reqs(10, seed=13, L_range=(60, 200), budget=(300, 600))
    specs = [dict(request_spec(r), stop_at_extinction=False) for r in reqs]
    srv = E.Server(arena_bytes=1 << 20, max_slots=4, keep_lattice=True, chunks_per_step=1)
    ids = [srv.submit(sp) for sp in specs]
    srv.step()                                   # a few runs resident, the rest queued
    resident, queued, _ = srv.stats()
    assert resident >= 1 and queued >= 1
    running, waiting = ids[0], ids[-1]
    srv.cancel(waiting)
    srv.step()
    srv.cancel(running)
    with pytest.raises(E.EscgError):
        srv.cancel(running)                      # already finished
    done = set()
    for _ in range(10000):
        done.update(srv.poll())
        if len(done) == len(ids):
            break
        srv.step()
    assert len(done) == len(ids)
    m, ext, cnt, lat = srv.result(waiting)
    assert m == 0 and not ext
    m, ext, cnt, lat = srv.result(running, lattice=True)
    sp = specs[0]
    assert 0 < m < sp["max_mcs"] and m % 10 == 0
    g = E.Lattice(sp["L"], sp["S"], sp["digraph"], sp["rates"], sp["seed"], p_empty=sp["p_empty"], log_every=10)
    g.run(m)
    assert np.array_equal(lat, g.snapshot())
    for rid, sp in zip(ids[1:-1], specs[1:-1]):
        m1, lat1, _ = _alone(sp)
        mcs, _, _, lat2 = srv.result(rid, lattice=True)
        assert mcs == m1 and np.array_equal(lat2, lat1), rid
    assert srv.stats() == (0, 0, 0)
