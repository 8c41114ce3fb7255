"""Pins of the random-sequential (RS) oracle -- Alg. 3 + Alg. 4 -- against
exact probability laws computed by brute force, and against invariants.

The rule table used by the brute force comes from the oracle's rule, which
is itself pinned by the paper's worked transitions (test_oracle_pins); what
is tested here is the sampling: a uniform cell, a uniform von Neumann
direction, an action drawn with probabilities epsilon/R, mu/R, sigma/R, and
N elementary steps per MCS on a periodic lattice.
"""
import numpy as np
import pytest
from scipy.stats import chisquare

import oracle as O

L3 = 3
NBR = {}


def _nbr(i, d, L=L3):
    r, c = divmod(i, L)
    if d == 0:
        r = (r - 1) % L
    elif d == 1:
        r = (r + 1) % L
    elif d == 2:
        c = (c - 1) % L
    else:
        c = (c + 1) % L
    return r * L + c


def _rule_table(D):
    S = D.shape[0]
    T = np.zeros((3, S + 1, S + 1, 2), dtype=np.int64)
    for act in range(3):
        for a in range(S + 1):
            for b in range(S + 1):
                T[act, a, b] = O.rule(act, a, b, D)
    return T


def _action_probs(I, P, X):
    R = X + I + P
    return np.array([X / R, I / R, P / R])


def test_periodic_neighbours_on_3x3_are_distinct():
    # on a 3x3 torus the four von Neumann neighbours are distinct sites
    for i in range(9):
        assert len({_nbr(i, d) for d in range(4)}) == 4


@pytest.mark.parametrize("rates", [(1.0, 1.0, 2.0), (1.0, 0.0, 0.0), (0.3, 1.7, 0.25)])
def test_one_step_law_3x3(rates):
    """Empirical distribution of the lattice after ONE elementary step equals
    the exact law (9 cells x 4 directions x 3 actions)."""
    I, P, X = rates
    D = O.circulant(3, [1])
    s0 = np.array([[1, 2, 0], [3, 1, 2], [0, 3, 3]], dtype=np.uint8)
    T = _rule_table(D)
    pa = _action_probs(I, P, X)
    exact = {}
    flat0 = s0.ravel()
    for i in range(9):
        for d in range(4):
            j = _nbr(i, d)
            for act in range(3):
                if pa[act] == 0:
                    continue
                s = flat0.copy()
                s[i], s[j] = T[act, s[i], s[j]]
                key = s.tobytes()
                exact[key] = exact.get(key, 0.0) + pa[act] / 36.0
    n = 60000
    emp = {}
    for k in range(n):
        lat = s0.copy()
        O.rs_attempts(lat, D, I, P, X, seed=0x5EED0000, n_attempts=1, stream=k)
        key = lat.ravel().tobytes()
        emp[key] = emp.get(key, 0) + 1
    assert set(emp) <= set(exact)
    keys = sorted(exact)
    f_obs = np.array([emp.get(k, 0) for k in keys], dtype=float)
    f_exp = np.array([exact[k] for k in keys]) * n
    assert abs(sum(exact.values()) - 1.0) < 1e-12
    assert chisquare(f_obs, f_exp).pvalue > 1e-3


def _exact_mcs_distribution(s0, D, I, P, X, n_attempts):
    """Exact distribution over all (S+1)^9 lattices after n_attempts steps."""
    S = D.shape[0]
    base = S + 1
    nstates = base ** 9
    codes = np.arange(nstates, dtype=np.int64)
    pw = base ** np.arange(9, dtype=np.int64)
    digits = (codes[:, None] // pw[None, :]) % base
    T = _rule_table(D)
    pa = _action_probs(I, P, X)
    p = np.zeros(nstates)
    p[int((s0.ravel().astype(np.int64) * pw).sum())] = 1.0
    moves = []
    for i in range(9):
        for d in range(4):
            j = _nbr(i, d)
            a, b = digits[:, i], digits[:, j]
            for act in range(3):
                if pa[act] == 0:
                    continue
                na, nb = T[act, a, b, 0], T[act, a, b, 1]
                new = codes + (na - a) * pw[i] + (nb - b) * pw[j]
                moves.append((new, pa[act] / 36.0))
    for _ in range(n_attempts):
        q = np.zeros(nstates)
        for new, w in moves:
            q += np.bincount(new, weights=p * w, minlength=nstates)
        p = q
    return p, digits


def test_one_mcs_brute_force_3x3():
    """One MCS = N = 9 elementary steps (Alg. 4).  The exact law of the count
    vector after one MCS, propagated over all 4^9 lattices, matches the RS
    oracle's empirical frequencies."""
    I, P, X = 1.0, 1.0, 0.5
    D = O.circulant(3, [1])
    s0 = np.array([[1, 2, 3], [0, 1, 2], [3, 0, 1]], dtype=np.uint8)
    p, digits = _exact_mcs_distribution(s0, D, I, P, X, 9)
    assert abs(p.sum() - 1) < 1e-9
    cnt = np.stack([(digits == v).sum(1) for v in range(4)], 1)
    cnt_code = cnt @ np.array([1, 10, 100, 1000])
    exact = {}
    nz = np.nonzero(p > 0)[0]
    for c, w in zip(cnt_code[nz], p[nz]):
        exact[int(c)] = exact.get(int(c), 0.0) + w
    n = 40000
    emp = {}
    for k in range(n):
        lat = O.rs_run(s0, D, I, P, X, seed=0xBEEF, n_mcs=1, stream=k)
        c = O.counts(lat, 3).astype(np.int64) @ np.array([1, 10, 100, 1000])
        emp[int(c)] = emp.get(int(c), 0) + 1
    assert set(emp) <= set(exact)
    keys = sorted(exact)
    f_exp = np.array([exact[k] for k in keys]) * n
    f_obs = np.array([emp.get(k, 0) for k in keys], dtype=float)
    # pool the rare outcomes into one bin so every bin expects >= 5
    rare = f_exp < 5
    f_exp = np.append(f_exp[~rare], f_exp[rare].sum())
    f_obs = np.append(f_obs[~rare], f_obs[rare].sum())
    if f_exp[-1] == 0:
        f_exp, f_obs = f_exp[:-1], f_obs[:-1]
    assert chisquare(f_obs, f_exp).pvalue > 1e-3


def test_exchange_destinations_uniform():
    """Cells and directions are uniform on a 5x5 torus: with exchange only, a
    single occupied cell moves to each of its 4 neighbours with equal
    probability."""
    L = 5
    D = O.circulant(3, [1])
    counts = np.zeros((L * L,), dtype=np.int64)
    moved = 0
    n = 25000
    for k in range(n):
        lat = np.zeros((L, L), dtype=np.uint8)
        lat[2, 2] = 1
        O.rs_attempts(lat, D, 0.0, 0.0, 1.0, seed=99, n_attempts=1, stream=k)
        idx = np.flatnonzero(lat.ravel())
        assert len(idx) == 1
        counts[idx[0]] += 1
        moved += idx[0] != 12
    # the occupied cell moves iff the drawn cell is it (1/25) or one of its 4
    # neighbours pointing at it (4 x 1/25 x 1/4): P(move) = 2/25, and each of
    # the 4 destinations gets 1/4 of the moves.
    dest = counts[[7, 17, 11, 13]]
    assert abs(moved / n - 2 / 25) < 4 * np.sqrt((2 / 25) * (23 / 25) / n)
    assert chisquare(dest).pvalue > 1e-3


@pytest.mark.parametrize("which", ["rs", "replay"])
def test_invariants(which):
    """Sum of counts = N; exchange-only conserves counts and permutes the
    lattice; monochrome and all-empty lattices are fixed points;
    competition-only never increases species or decreases empties;
    reproduction-only never increases empties."""
    L, S = 16, 3
    D = O.circulant(S, [1])
    N = L * L

    def run(lat, I, P, X, n_mcs, seed):
        if which == "rs":
            return O.rs_run(lat, D, I, P, X, seed, n_mcs)
        return O.replay_run(lat, D, I, P, X, seed, n_mcs)[0]

    lat0 = O.init(L, S, 0.25, 11)
    # exchange only
    lat = run(lat0, 0.0, 0.0, 1.0, 5, 1)
    assert np.array_equal(np.sort(lat.ravel()), np.sort(lat0.ravel()))
    assert not np.array_equal(lat, lat0)
    # fixed points
    for v in range(S + 1):
        mono = np.full((L, L), v, dtype=np.uint8)
        assert np.array_equal(run(mono, 1.0, 1.0, 3.0, 3, 2), mono)
    # competition only
    prev = O.counts(lat0, S)
    lat = lat0
    for k in range(5):
        lat = run(lat, 1.0, 0.0, 0.0, 1, 3 + k) if which == "rs" else \
            O.replay_run(lat, D, 1.0, 0.0, 0.0, 3, 1, mcs_begin=k)[0]
        c = O.counts(lat, S)
        assert c.sum() == N
        assert c[0] >= prev[0] and (c[1:] <= prev[1:]).all()
        prev = c
    # reproduction only
    prev = O.counts(lat0, S)
    lat = lat0
    for k in range(5):
        lat = run(lat, 0.0, 1.0, 0.0, 1, 30 + k) if which == "rs" else \
            O.replay_run(lat, D, 0.0, 1.0, 0.0, 30, 1, mcs_begin=k)[0]
        c = O.counts(lat, S)
        assert c.sum() == N and c[0] <= prev[0] and (c[1:] >= prev[1:]).all()
        prev = c
