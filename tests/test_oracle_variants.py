"""Pins of the rule variants of both oracles: the paper's 8-way (Moore)
neighbourhood and its non-wrapping boundary (Alg. 3: a direction from
[0, neighbourhood), the neighbour "updated using dir and boundary conditions",
"flux or reflect"; the CLI's --neighbourhood and --flux options).

Pinned against: exact one-attempt laws of the random-sequential oracle that
tell the variants apart (3x3 lattices, closed-form probabilities); the
schedule's structure on full traces (neighbour at Chebyshev distance 1 in
the drawn direction, mirrored at the edge; uniform directions; race freedom
inside every coarse and fine phase); and random-sequential dynamics (mean
densities over seeds).
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O

DR = np.array([-1, 1, 0, 0, -1, -1, 1, 1])
DC = np.array([0, 0, -1, 1, -1, 1, -1, 1])
ONE_BEATS_TWO = np.array([[0, 1], [0, 0]], dtype=np.uint8)


def _death_rate(lat0, n=9000, **kw):
    """Fraction of single interaction attempts that empty the species-2 cell."""
    r, c = np.argwhere(lat0 == 2)[0]
    deaths = 0
    for s in range(n):
        lat = O.rs_attempts(lat0.copy(), ONE_BEATS_TWO, 1.0, 0.0, 0.0, 7000 + s, 1, **kw)
        deaths += int(lat[r, c] == 0)
    return deaths / n, n


def _close(rate, n, q):
    return abs(rate - q) < 4 * np.sqrt(q * (1 - q) / n)


def test_moore_one_attempt_law():
    """Species 2 at the centre of a 3x3 torus, species 1 on the four
    diagonal cells only: Moore contact is diagonal, so P(death) =
    (1/9)(4/8) + 4 (1/9)(1/8) = 1/9; the von Neumann neighbourhood never
    reaches it (0)."""
    lat0 = np.zeros((3, 3), dtype=np.uint8)
    lat0[1, 1] = 2
    for r, c in [(0, 0), (0, 2), (2, 0), (2, 2)]:
        lat0[r, c] = 1
    rate, n = _death_rate(lat0, neighbourhood=8)
    assert _close(rate, n, 1 / 9), rate
    rate4, _ = _death_rate(lat0, n=2000, neighbourhood=4)
    assert rate4 == 0.0


def test_reflecting_boundary_one_attempt_law():
    """Species 2 in the corner (0, 0) of a 3x3 lattice, species 1 at (0, 1)
    and (1, 0): with reflection every step from the corner meets species 1
    (up mirrors to down, left to right), so P(death) = 1/9 + 2 (1/9)(1/4) =
    1/6; with wrap-around only two of the four steps do, P = 1/9."""
    lat0 = np.zeros((3, 3), dtype=np.uint8)
    lat0[0, 0] = 2
    lat0[0, 1] = lat0[1, 0] = 1
    rate, n = _death_rate(lat0, reflect=True)
    assert _close(rate, n, 1 / 6), rate
    rate_w, n_w = _death_rate(lat0, reflect=False)
    assert _close(rate_w, n_w, 1 / 9), rate_w


def test_default_variant_is_the_original_rule():
    D = O.circulant(3, (1,))
    lat = O.init(40, 3, 0.2, 3)
    a, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, 3, 3)
    b, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, 3, 3, neighbourhood=4, reflect=False)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("L,nbh,reflect", [(24, 8, False), (19, 4, True), (33, 8, True), (64, 8, False)])
def test_trace_neighbours_directions_and_race_freedom(L, nbh, reflect):
    D = O.circulant(5, (1, 2))
    lat0 = O.init(L, 5, 0.2, 8)
    nmcs = 2
    lat, att, tr = O.replay_run(lat0, D, 1.0, 1.0, 1.0, 21, nmcs, trace_cap=L * L * nmcs + 1,
                                neighbourhood=nbh, reflect=reflect)
    assert att == L * L * nmcs
    site, nbr = tr["site"].astype(np.int64), tr["nbr"].astype(np.int64)
    r, c = site // L, site % L
    nr, nc = nbr // L, nbr % L
    d = tr["dir"].astype(int)
    assert (d < nbh).all()
    er, ec = r + DR[d], c + DC[d]
    if reflect:
        er = np.where((er < 0) | (er >= L), r - DR[d], er)
        ec = np.where((ec < 0) | (ec >= L), c - DC[d], ec)
        assert (np.abs(nr - r) <= 1).all() and (np.abs(nc - c) <= 1).all()
    else:
        er, ec = er % L, ec % L
    assert (nr == er).all() and (nc == ec).all()
    # directions uniform over the neighbourhood (chi-square, 8 or 4 cells)
    cnt = np.bincount(d, minlength=nbh)
    exp = len(d) / nbh
    assert ((cnt - exp) ** 2 / exp).sum() < 40
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


def _dens(args):
    use_rs, seed, nbh, reflect = args
    S, L, n = 3, 32, 30
    D = O.circulant(S, (1,))
    lat = O.init(L, S, 0.25, seed)
    if use_rs:
        lat = O.rs_run(lat, D, 1.0, 1.0, 2.0, seed ^ 0x3C3C3C3C, n, neighbourhood=nbh, reflect=reflect)
    else:
        lat, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, seed, n, neighbourhood=nbh, reflect=reflect)
    return O.counts(lat, S) / (L * L)


@pytest.mark.parametrize("nbh,reflect", [(8, False), (4, True), (8, True)])
def test_replay_schedule_matches_random_sequential_for_variants(nbh, reflect):
    seeds = [0x5EED2000 + i for i in range(48)]
    with mp.get_context("spawn").Pool(8) as pool:
        rs = np.array(pool.map(_dens, [(True, s, nbh, reflect) for s in seeds]))
        rp = np.array(pool.map(_dens, [(False, s, nbh, reflect) for s in seeds]))
    se = np.sqrt(rs.var(axis=0, ddof=1) / len(seeds) + rp.var(axis=0, ddof=1) / len(seeds))
    assert np.all(np.abs(rs.mean(axis=0) - rp.mean(axis=0)) < 3 * se + 1e-12)
