"""Pins of the schedule-v1 replay oracle.

The replay oracle executes the coloured two-level sublattice schedule
serially.  Its correctness is pinned by properties the schedule's definition
fixes, checked on a full trace of every elementary step:

* the partition (coarse P even, fine Q even per coarse segment, widths);
* exactly N = L^2 elementary steps per MCS (Alg. 4), each sub-block k taking
  attempts t = 0..n_k-1 exactly once;
* every attempt's cell lies in its own sub-block and its neighbour is the
  periodic von Neumann neighbour in the drawn direction (Section 3.1);
* race freedom: inside a coarse phase the sites touched by different blocks
  are disjoint, and inside a fine phase the sites touched by different
  sub-blocks are disjoint -- hence the result cannot depend on the order in
  which a phase's independent units run, which is also checked directly;
* uniform draws of the cell within a sub-block, of the direction, of the
  colour orders, and action frequencies equal to the rate thresholds.
"""
import itertools

import numpy as np
import pytest
from scipy.stats import chisquare

import oracle as O


def _nbr(L, i, d):
    r, c = divmod(int(i), L)
    if d == 0:
        r = (r - 1) % L
    elif d == 1:
        r = (r + 1) % L
    elif d == 2:
        c = (c - 1) % L
    else:
        c = (c + 1) % L
    return r * L + c


@pytest.mark.parametrize("L", list(range(8, 140)) + [199, 200, 400, 401, 777, 800, 1600, 3200, 3201])
def test_partition(L):
    cs, fs, fc = O.v1_partition(L)
    P = len(cs) - 1
    assert P % 2 == 0 and P >= 2
    w = np.diff(cs)
    assert cs[0] == 0 and cs[-1] == L and w.max() - w.min() <= 1
    GQ = len(fs) - 1
    assert fs[0] == 0 and fs[-1] == L and fc[-1] == GQ
    for k in range(P):
        Q = fc[k + 1] - fc[k]
        assert Q % 2 == 0 and Q >= 2
        seg = fs[fc[k]:fc[k + 1] + 1]
        assert seg[0] == cs[k] and seg[-1] == cs[k + 1]
        fw = np.diff(seg)
        assert fw.min() >= 2 and fw.max() <= 4 and fw.max() - fw.min() <= 1
    if L == 3200:
        assert P == 50 and (w == 64).all() and (np.diff(fs) == 2).all()
    if L == 64:
        assert P == 2 and (w == 32).all() and (np.diff(fs) == 2).all()


def _subblock_of(fs, GQ):
    """site coordinate -> global fine index along one axis"""
    idx = np.zeros(fs[-1], dtype=np.int64)
    for g in range(GQ):
        idx[fs[g]:fs[g + 1]] = g
    return idx


@pytest.mark.parametrize("L,S,rates,nmcs", [(8, 3, (1, 1, 1), 3), (13, 3, (1, 1, 0.5), 2),
                                            (20, 5, (1, 1, 2), 2), (64, 3, (1, 0, 0), 2),
                                            (67, 5, (1, 1, 3), 1)])
def test_trace_structure_and_race_freedom(L, S, rates, nmcs):
    I, P, X = rates
    D = O.circulant(S, [1] if S == 3 else [1, 2])
    cs, fs, fc = O.v1_partition(L)
    Pc, GQ = len(cs) - 1, len(fs) - 1
    N = L * L
    lat0 = O.init(L, S, 0.2, 5)
    lat, att, tr = O.replay_run(lat0, D, I, P, X, 77, nmcs, trace_cap=N * nmcs + 1)
    assert att == N * nmcs and len(tr) == N * nmcs
    fine_of = _subblock_of(fs, GQ)
    coarse_of = np.zeros(L, dtype=np.int64)
    for k in range(Pc):
        coarse_of[cs[k]:cs[k + 1]] = k
    rows, cols = tr["site"] // L, tr["site"] % L
    # cell inside its own sub-block and its own block
    assert (fine_of[rows] * GQ + fine_of[cols] == tr["sub"]).all()
    assert (coarse_of[rows] * Pc + coarse_of[cols] == tr["block"]).all()
    # neighbour = periodic von Neumann neighbour in direction dir
    nb = np.array([_nbr(L, s, d) for s, d in zip(tr["site"], tr["dir"])])
    assert (nb == tr["nbr"]).all()
    # every sub-block takes t = 0..n_k-1 exactly once per MCS
    wid = np.diff(fs)
    for m in range(nmcs):
        sel = tr[tr["mcs"] == m]
        assert len(sel) == N
        gy, gx = sel["sub"] // GQ, sel["sub"] % GQ
        nk = wid[gy] * wid[gx]
        key = sel["sub"].astype(np.int64) * 64 + sel["t"]
        assert len(np.unique(key)) == N
        assert (sel["t"] < nk).all()
        # one coarse phase per colour, each block visited once per MCS
        phases = np.unique(sel["coarse_phase"])
        assert len(phases) == 4
        colours = []
        for ph in phases:
            blk = np.unique(sel["block"][sel["coarse_phase"] == ph])
            col = {2 * ((b // Pc) % 2) + (b % Pc) % 2 for b in blk}
            assert len(col) == 1
            colours.append(col.pop())
            assert len(blk) == (Pc * Pc) // 4
        assert sorted(colours) == [0, 1, 2, 3]
    # race freedom inside every coarse phase and every fine phase
    for key_name, unit in [("coarse_phase", "block"), ("fine_phase", "sub")]:
        for ph in np.unique(tr[key_name]):
            sel = tr[tr[key_name] == ph]
            owner = {}
            for u, s, n in zip(sel[unit], sel["site"], sel["nbr"]):
                for x in (int(s), int(n)):
                    assert owner.setdefault(x, int(u)) == int(u), (key_name, ph, x)
    # the final lattice of the traced run equals an untraced run
    lat2, _ = O.replay_run(lat0, D, I, P, X, 77, nmcs)
    assert np.array_equal(lat, lat2)


@pytest.mark.parametrize("L", [8, 13, 50, 64, 100, 131])
def test_order_independence_within_phases(L):
    """Permuting the blocks of each coarse phase and the sub-blocks of each
    fine phase never changes the lattice (the schedule is race-free)."""
    S = 5
    D = O.circulant(S, [1, 2])
    lat0 = O.init(L, S, 1.0 / 6, 1234 + L)
    ref, _ = O.replay_run(lat0, D, 1.0, 1.0, 2.0, 42, 3)
    for k in range(3):
        got, _ = O.replay_run(lat0, D, 1.0, 1.0, 2.0, 42, 3,
                              flags=O.SHUFFLE_BLOCKS | O.SHUFFLE_SUBS, shuffle_seed=k + 1)
        assert np.array_equal(got, ref)


def test_draw_frequencies():
    """Cell within the sub-block, direction and action are drawn with the
    stated probabilities; the 24 coarse colour orders are uniform."""
    L, S = 16, 3
    D = O.circulant(S, [1])
    I, P, X = 1.0, 1.0, 2.0
    nmcs = 200
    lat0 = O.init(L, S, 0.25, 3)
    _, att, tr = O.replay_run(lat0, D, I, P, X, 9, nmcs, trace_cap=L * L * nmcs)
    cs, fs, fc = O.v1_partition(L)
    GQ = len(fs) - 1
    assert (np.diff(fs) == 2).all()
    gy, gx = tr["sub"] // GQ, tr["sub"] % GQ
    local = (tr["site"] // L - fs[gy]) * 2 + (tr["site"] % L - fs[gx])
    assert chisquare(np.bincount(local, minlength=4)).pvalue > 1e-3
    assert chisquare(np.bincount(tr["dir"], minlength=4)).pvalue > 1e-3
    # joint (cell, direction) uniform too
    assert chisquare(np.bincount(local * 4 + tr["dir"], minlength=16)).pvalue > 1e-3
    # actions: only attempts on distinct pairs are classified by the trace,
    # and the action is recorded for all of them
    n = len(tr)
    for act, p in [(0, X / (X + I + P)), (1, I / (X + I + P)), (2, P / (X + I + P))]:
        k = (tr["action"] == act).sum()
        assert abs(k / n - p) < 5 * np.sqrt(p * (1 - p) / n)
    # coarse colour order per MCS: uniform over the 24 permutations
    nmcs2 = 2400
    _, _, tr2 = O.replay_run(O.init(8, S, 0.25, 4), D, I, P, X, 11, nmcs2, trace_cap=64 * nmcs2)
    cs8, _, _ = O.v1_partition(8)
    Pc = len(cs8) - 1
    perms = {p: i for i, p in enumerate(itertools.permutations(range(4)))}
    idx = []
    for m in range(nmcs2):
        sel = tr2[tr2["mcs"] == m]
        order = []
        for ph in np.unique(sel["coarse_phase"]):
            b = sel["block"][sel["coarse_phase"] == ph][0]
            order.append(2 * ((b // Pc) % 2) + (b % Pc) % 2)
        idx.append(perms[tuple(order)])
    assert chisquare(np.bincount(idx, minlength=24)).pvalue > 1e-3


@pytest.mark.parametrize("S,p_empty", [(3, 0.0), (3, 0.25), (5, 0.2), (5, 1.0), (7, 0.5)])
def test_init_distribution(S, p_empty):
    L = 200
    lat = O.init(L, S, p_empty, 31337)
    c = O.counts(lat, S).astype(float)
    N = L * L
    assert abs(c[0] / N - p_empty) < 5 * np.sqrt(max(p_empty * (1 - p_empty), 1e-12) / N) + 1e-12
    if p_empty < 1:
        assert chisquare(c[1:]).pvalue > 1e-3
    # deterministic in the seed, different across seeds
    assert np.array_equal(lat, O.init(L, S, p_empty, 31337))
    if 0 < p_empty < 1:
        assert not np.array_equal(lat, O.init(L, S, p_empty, 31338))


def test_resume_is_exact():
    """run(a + b) == run(a) followed by run(b) from MCS a (counter-based
    randomness keyed by the absolute MCS number)."""
    L, S = 40, 3
    D = O.circulant(S, [1])
    lat0 = O.init(L, S, 0.25, 8)
    full, _ = O.replay_run(lat0, D, 1, 1, 0.8, 8, 7)
    part, _ = O.replay_run(lat0, D, 1, 1, 0.8, 8, 3)
    rest, _ = O.replay_run(part, D, 1, 1, 0.8, 8, 4, mcs_begin=3)
    assert np.array_equal(full, rest)
    rs_full = O.rs_run(lat0, D, 1, 1, 0.8, 8, 5)
    rs_rest = O.rs_run(O.rs_run(lat0, D, 1, 1, 0.8, 8, 2), D, 1, 1, 0.8, 8, 3, mcs_begin=2)
    assert np.array_equal(rs_full, rs_rest)


def test_observed_run_logging_and_stasis():
    """Counts logged at every multiple of log_every (including MCS 0); a run
    with stop_at_extinction ends at the first logged MCS with <= 1 species."""
    L, S = 16, 3
    D = O.circulant(S, [1])
    lat0 = O.init(L, S, 0.25, 2)
    lat, log, mend = O.run_observed(lat0, D, 1.0, 1.0, 0.0, 2, 20, log_every=5)
    assert mend == 20 and len(log) == 5
    assert (log.sum(1) == L * L).all()
    ref, _ = O.replay_run(lat0, D, 1.0, 1.0, 0.0, 2, 20)
    assert np.array_equal(lat, ref)
    assert np.array_equal(log[-1], O.counts(ref, S))
    # a lattice with one species (plus empties) stops immediately
    mono = np.where(lat0 > 0, 1, 0).astype(np.uint8)
    _, log2, mend2 = O.run_observed(mono, D, 1.0, 1.0, 0.0, 2, 20, log_every=5,
                                    stop_at_extinction=True)
    assert mend2 == 0 and len(log2) == 1
    # high mobility on a small lattice goes extinct well within the budget
    lat3, log3, mend3 = O.run_observed(O.init(8, S, 0.25, 3), D, 1.0, 1.0, 64.0, 3, 5000,
                                       log_every=10, stop_at_extinction=True)
    assert mend3 % 10 == 0 and mend3 < 5000
    assert (O.counts(lat3, S)[1:] > 0).sum() <= 1
    assert ((log3[:-1, 1:] > 0).sum(1) >= 2).all()
