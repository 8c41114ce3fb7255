"""Pins of the probabilistic-dominance extension of both oracles (Park, Chen
and Szolnoki's model as the paper's section "Park, Chen, Szolnoki" describes
it: every edge of the dominance network carries the probability that an
interaction across it takes place; mobility is optional).

Pinned against: the deterministic model (every probability 1) and the model
with an edge removed (its probability 0), bit for bit; the closed form of the
schedule's integer threshold; the exact one-attempt law of the
random-sequential oracle on a 3x3 torus; and the random-sequential dynamics
for the replay schedule (mean densities over seeds).
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O


def _prob(S, D, value):
    P = np.zeros((S, S))
    P[D.astype(bool)] = value
    return P


@pytest.mark.parametrize("S,K", [(3, (1,)), (5, (1, 2))])
def test_probability_one_is_the_deterministic_model(S, K):
    D = O.circulant(S, K)
    lat = O.init(40, S, 0.2, 11)
    a, _ = O.replay_run(lat, D, 1.0, 1.0, 3.0, 11, 3)
    b, _ = O.replay_run(lat, D, 1.0, 1.0, 3.0, 11, 3, prob=_prob(S, D, 1.0))
    assert np.array_equal(a, b)
    c = O.rs_run(lat, D, 1.0, 1.0, 3.0, 11, 2)
    e = O.rs_run(lat, D, 1.0, 1.0, 3.0, 11, 2, prob=_prob(S, D, 1.0))
    assert np.array_equal(c, e)


def test_probability_zero_removes_the_edge():
    S = 5
    D = O.circulant(S, (1, 2))
    P = _prob(S, D, 1.0)
    P[0, 2] = 0.0                        # species 1 never beats species 3
    Dr = D.copy()
    Dr[0, 2] = 0
    lat = O.init(48, S, 0.2, 5)
    a, _ = O.replay_run(lat, D, 1.0, 1.0, 1.0, 5, 4, prob=P)
    b, _ = O.replay_run(lat, Dr, 1.0, 1.0, 1.0, 5, 4)
    assert np.array_equal(a, b)
    c = O.rs_run(lat, D, 1.0, 1.0, 1.0, 5, 2, prob=P)
    e = O.rs_run(lat, Dr, 1.0, 1.0, 1.0, 5, 2)
    assert np.array_equal(c, e)


def test_interaction_threshold_closed_form():
    T = O.interaction_threshold
    assert T(0, 2**31, 0.25) == 2**29
    assert T(0, 2**32, 0.5) == 2**31
    assert T(1000, 5000, 0.0) == 1000 and T(1000, 5000, 1.0) == 5000
    # round(4000 * round(0.3 * 2^32) / 2^32) = 1200
    assert T(1000, 5000, 0.3) == 2200
    ts = [T(123, 2**32, p) for p in np.linspace(0, 1, 101)]
    assert all(x <= y for x, y in zip(ts, ts[1:]))


def test_pair_probability_is_the_edge_between_the_pair():
    D = O.circulant(3, (1,))            # 1 -> 2 -> 3 -> 1
    P = np.array([[0, 0.3, 0], [0, 0, 0.6], [0.9, 0, 0]])
    assert O.pair_prob(1, 2, D, P) == pytest.approx(0.3)
    assert O.pair_prob(2, 1, D, P) == pytest.approx(0.3)
    assert O.pair_prob(3, 2, D, P) == pytest.approx(0.6)
    assert O.pair_prob(1, 3, D, P) == pytest.approx(0.9)
    assert O.pair_prob(1, 0, D, P) == 1.0 and O.pair_prob(2, 2, D, P) == 1.0


@pytest.mark.parametrize("p", [0.2, 0.7])
def test_random_sequential_one_attempt_law(p):
    """3x3 torus of species 1 with one species-2 cell, interaction only: one
    attempt involves the species-2 cell with probability 2/9 (it is selected,
    or one of its 4 neighbours is selected with the direction towards it), and
    then kills it with probability p: P(death) = 2p/9 exactly."""
    D = np.array([[0, 1], [0, 0]], dtype=np.uint8)   # 1 beats 2, not the reverse
    P = np.array([[0.0, p], [0.0, 0.0]])
    lat0 = np.ones((3, 3), dtype=np.uint8)
    lat0[1, 1] = 2
    n, deaths = 6000, 0
    for s in range(n):
        lat = O.rs_attempts(lat0.copy(), D, 1.0, 0.0, 0.0, 1000 + s, 1, prob=P)
        deaths += int(lat[1, 1] == 0)
    q = 2 * p / 9
    sd = np.sqrt(n * q * (1 - q))
    assert abs(deaths - n * q) < 4 * sd, (deaths, n * q)


def _dens(args):
    use_rs, seed, prob = args
    S, L, n = 3, 32, 30
    D = O.circulant(S, (1,))
    lat = O.init(L, S, 0.25, seed)
    if use_rs:
        lat = O.rs_run(lat, D, 1.0, 1.0, 2.0, seed ^ 0x5A5A5A5A, n, prob=prob)
    else:
        lat, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, seed, n, prob=prob)
    return O.counts(lat, S) / (L * L)


def test_replay_schedule_matches_random_sequential_with_edge_probabilities():
    """Mean densities after 30 MCS over 48 seeds agree within 3 standard
    errors; the same comparison separates p = 0.3 from p = 1 by far more."""
    S = 3
    D = O.circulant(S, (1,))
    P = _prob(S, D, 0.3)
    seeds = [0x5EED1000 + i for i in range(48)]
    with mp.get_context("spawn").Pool(8) as pool:
        rs = np.array(pool.map(_dens, [(True, s, P) for s in seeds]))
        rp = np.array(pool.map(_dens, [(False, s, P) for s in seeds]))
        det = np.array(pool.map(_dens, [(False, s, None) for s in seeds]))
    se = np.sqrt(rs.var(axis=0, ddof=1) / len(seeds) + rp.var(axis=0, ddof=1) / len(seeds))
    assert np.all(np.abs(rs.mean(axis=0) - rp.mean(axis=0)) < 3 * se + 1e-12)
    # sensitivity: the empty density differs strongly from the deterministic model
    se_d = np.sqrt(rp.var(axis=0, ddof=1) / len(seeds) + det.var(axis=0, ddof=1) / len(seeds))
    assert abs(rp.mean(axis=0)[0] - det.mean(axis=0)[0]) > 6 * se_d[0]
