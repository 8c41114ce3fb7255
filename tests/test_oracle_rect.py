"""Pins of rectangular lattices in both oracles: L columns by H rows (the
paper's --length and --height options; Alg. 3 and 4 with N = L*H sites).

Pinned against: the square lattice (H = L) bit for bit; the counter-based
initial state (site i of an L x H lattice is site i of any lattice with the
same seed); the schedule's structure on full traces (each axis partitioned on
its own, every sub-block performing as many attempts per MCS as it has
cells, neighbours wrapped or mirrored on an H x L torus, race freedom inside
every coarse and fine phase); and random-sequential dynamics (mean densities
over seeds).
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O

DR = np.array([-1, 1, 0, 0, -1, -1, 1, 1])
DC = np.array([0, 0, -1, 1, -1, 1, -1, 1])


def test_square_is_the_default_height():
    D = O.circulant(3, (1,))
    a = O.init(40, 3, 0.2, 5)
    b = O.init(40, 3, 0.2, 5, H=40)
    assert np.array_equal(a, b)
    x, _ = O.replay_run(a, D, 1.0, 1.0, 2.0, 5, 3)
    y, _ = O.replay_run(b, D, 1.0, 1.0, 2.0, 5, 3, neighbourhood=4)
    assert np.array_equal(x, y)


def test_initial_state_is_indexed_by_site():
    """The initial species of site i is a function of (seed, i) only."""
    big = O.init(60, 4, 0.3, 77, H=50)
    assert big.shape == (50, 60)
    flat = big.reshape(-1)
    for L, H in [(30, 17), (60, 9), (100, 3)]:
        r = O.init(L, 4, 0.3, 77, H=H).reshape(-1)
        assert np.array_equal(r, flat[:L * H])
    # empty fraction and uniform species among occupied sites
    c = O.counts(O.init(400, 3, 0.25, 3, H=250), 3) / 1e5
    assert abs(c[0] - 0.25) < 0.005
    assert np.all(np.abs(c[1:] - 0.25) < 0.006)


@pytest.mark.parametrize("L,H,nbh,reflect", [(40, 24, 4, False), (24, 57, 8, False), (33, 70, 4, True),
                                             (136, 20, 8, True)])
def test_trace_partition_neighbours_and_race_freedom(L, H, nbh, reflect):
    D = O.circulant(5, (1, 2))
    lat0 = O.init(L, 5, 0.2, 8, H=H)
    nmcs = 2
    lat, att, tr = O.replay_run(lat0, D, 1.0, 1.0, 1.0, 21, nmcs, trace_cap=L * H * nmcs + 1,
                                neighbourhood=nbh, reflect=reflect)
    assert att == L * H * nmcs
    site, nbr = tr["site"].astype(np.int64), tr["nbr"].astype(np.int64)
    r, c = site // L, site % L
    assert (r < H).all()
    nr, nc = nbr // L, nbr % L
    d = tr["dir"].astype(int)
    er, ec = r + DR[d], c + DC[d]
    if reflect:
        er = np.where((er < 0) | (er >= H), r - DR[d], er)
        ec = np.where((ec < 0) | (ec >= L), c - DC[d], ec)
    else:
        er, ec = er % H, ec % L
    assert (nr == er).all() and (nc == ec).all()
    # the sub-blocks are the products of each axis's own fine partition
    _, fs, _ = O.v1_partition(L)
    _, rfs, _ = O.v1_partition(H)
    GQ = len(fs) - 1
    gy, gx = tr["sub"] // GQ, tr["sub"] % GQ
    assert (gy < len(rfs) - 1).all()
    assert ((r >= rfs[gy]) & (r < rfs[gy + 1]) & (c >= fs[gx]) & (c < fs[gx + 1])).all()
    # every sub-block performs as many attempts per MCS as it has cells
    area = (rfs[gy + 1] - rfs[gy]) * (fs[gx + 1] - fs[gx])
    for m in range(nmcs):
        sel = tr["mcs"] == m
        subs, cnt = np.unique(tr["sub"][sel], return_counts=True)
        assert len(subs) == GQ * (len(rfs) - 1)
        a = dict(zip(tr["sub"][sel], area[sel]))
        assert all(a[s] == k for s, k in zip(subs, cnt))
    # race freedom inside every coarse phase and every fine phase
    for key_name, unit in [("coarse_phase", "block"), ("fine_phase", "sub")]:
        for ph in np.unique(tr[key_name]):
            sel = tr[tr[key_name] == ph]
            owner = {}
            for u, s, n in zip(sel[unit], sel["site"], sel["nbr"]):
                for x in (int(s), int(n)):
                    assert owner.setdefault(x, int(u)) == int(u), (key_name, ph, x)
    lat2, _ = O.replay_run(lat0, D, 1.0, 1.0, 1.0, 21, nmcs, neighbourhood=nbh, reflect=reflect)
    assert np.array_equal(lat, lat2)


def test_run_observed_counts_every_site():
    D = O.circulant(3, (1,))
    lat = O.init(48, 3, 0.2, 4, H=20)
    out, log, mend = O.run_observed(lat, D, 1.0, 1.0, 2.0, 4, 6, log_every=2)
    assert mend == 6 and log.shape == (4, 4)
    assert (log.sum(axis=1) == 48 * 20).all()
    assert np.array_equal(log[-1], O.counts(out, 3))
    assert np.array_equal(log[0], O.counts(lat, 3))


def _dens(args):
    use_rs, seed = args
    S, L, H, n = 3, 48, 24, 30
    D = O.circulant(S, (1,))
    lat = O.init(L, S, 0.25, seed, H=H)
    if use_rs:
        lat = O.rs_run(lat, D, 1.0, 1.0, 2.0, seed ^ 0x0F0F0F0F, n)
    else:
        lat, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, seed, n)
    return O.counts(lat, S) / (L * H)


def test_replay_schedule_matches_random_sequential_on_a_rectangle():
    seeds = [0x5EED3000 + i for i in range(48)]
    with mp.get_context("spawn").Pool(8) as pool:
        rs = np.array(pool.map(_dens, [(True, s) for s in seeds]))
        rp = np.array(pool.map(_dens, [(False, s) for s in seeds]))
    se = np.sqrt(rs.var(axis=0, ddof=1) / len(seeds) + rp.var(axis=0, ddof=1) / len(seeds))
    assert np.all(np.abs(rs.mean(axis=0) - rp.mean(axis=0)) < 3 * se + 1e-12)
