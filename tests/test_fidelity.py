"""Statistical fidelity of the coloured-sublattice schedule (version 1) to
true random-sequential dynamics (Alg. 3 + Alg. 4).

The schedule is a declared approximation of the random-sequential process:
it replaces "N attempts at uniformly random sites, one after another" by a
race-free parallel order.  These tests compare the replay oracle (which the
GPU path reproduces bit for bit) with the random-sequential oracle over 64
seeds: mean species densities at several MCS must agree within three
standard errors of the difference, and extinction probabilities within
their binomial (Wilson) 95% intervals.

Both oracles are CPU code; the comparison runs in a process pool.
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O

NSEEDS = 64
SEED0 = 0x5EED0000


def _densities(args):
    use_rs, L, S, K, p_empty, I, P, M, seed, checkpoints = args
    D = O.circulant(S, K)
    N = L * L
    X = O.exchange_from_mobility(M, N)
    lat = O.init(L, S, p_empty, seed)
    out, m = [], 0
    for c in checkpoints:
        if use_rs:
            lat = O.rs_run(lat, D, I, P, X, seed ^ 0xA5A5A5A5, c - m, mcs_begin=m)
        else:
            lat, _ = O.replay_run(lat, D, I, P, X, seed, c - m, mcs_begin=m)
        m = c
        out.append(O.counts(lat, S) / N)
    return np.array(out)


@pytest.fixture(scope="module")
def pool():
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, max(2, mp.cpu_count()))) as p:
        yield p


CASES = [
    # (name, L, S, K, p_empty, I, P, M, checkpoints)
    ("rps-competition-only-L64", 64, 3, [1], 0.0, 1.0, 0.0, 0.0, [10, 100]),
    ("rpsls-80pct-occupied-L64-M1e-4", 64, 5, [1, 2], 0.2, 1.0, 1.0, 1e-4, [10, 100, 1000]),
    ("rps-uniform-L100-M1e-4", 100, 3, [1], 0.25, 1.0, 1.0, 1e-4, [10, 100, 1000]),
    ("rps-uniform-L100-M1e-3", 100, 3, [1], 0.25, 1.0, 1.0, 1e-3, [10, 100, 1000]),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_mean_densities_agree_with_random_sequential(pool, case):
    name, L, S, K, p_empty, I, P, M, cps = case
    rs = np.array(pool.map(_densities, [(1, L, S, K, p_empty, I, P, M, SEED0 + s, cps)
                                        for s in range(NSEEDS)]))
    rp = np.array(pool.map(_densities, [(0, L, S, K, p_empty, I, P, M, SEED0 + s, cps)
                                        for s in range(NSEEDS)]))
    diff = rp.mean(0) - rs.mean(0)
    se = np.sqrt(rp.var(0, ddof=1) / NSEEDS + rs.var(0, ddof=1) / NSEEDS)
    z = np.abs(diff) / np.where(se > 0, se, 1.0)
    assert (z < 3.0).all(), f"{name}: |z| per checkpoint/state =\n{np.round(z, 2)}"
    # and both conserve the site count
    assert np.allclose(rs.sum(2), 1.0) and np.allclose(rp.sum(2), 1.0)


def _extinction_mcs(args):
    use_rs, L, S, K, M, seed, budget = args
    D = O.circulant(S, K)
    X = O.exchange_from_mobility(M, L * L)
    lat = O.init(L, S, 1.0 / (S + 1), seed)
    _, _, mend = O.run_observed(lat, D, 1.0, 1.0, X, seed, budget, log_every=10,
                                stop_at_extinction=True, use_rs=bool(use_rs))
    return mend


def _wilson(k, n, z=1.96):
    p = k / n
    den = 1 + z * z / n
    c = (p + z * z / (2 * n)) / den
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return c - h, c + h


EXT_CASES = [
    # (name, L, S, K, M, budget)
    # budgets near the median extinction time, so the probability is
    # intermediate and the comparison discriminates
    ("rps-L64-M3e-4", 64, 3, [1], 3e-4, 3000),
    ("rpsls-L64-M1e-3", 64, 5, [1, 2], 1e-3, 1000),
]


@pytest.mark.parametrize("case", EXT_CASES, ids=[c[0] for c in EXT_CASES])
def test_extinction_probability_agrees(pool, case):
    name, L, S, K, M, budget = case
    rs = np.array(pool.map(_extinction_mcs, [(1, L, S, K, M, SEED0 + s, budget) for s in range(NSEEDS)]))
    rp = np.array(pool.map(_extinction_mcs, [(0, L, S, K, M, SEED0 + s, budget) for s in range(NSEEDS)]))
    k_rs, k_rp = int((rs < budget).sum()), int((rp < budget).sum())
    lo_rs, hi_rs = _wilson(k_rs, NSEEDS)
    lo_rp, hi_rp = _wilson(k_rp, NSEEDS)
    # each estimate lies inside the other's 95% interval
    assert lo_rs <= k_rp / NSEEDS <= hi_rs, (name, k_rs, k_rp)
    assert lo_rp <= k_rs / NSEEDS <= hi_rp, (name, k_rs, k_rp)
