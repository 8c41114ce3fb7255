"""Seeded synthetic workloads shaped like the paper's (no dataset exists:
every ESCG workload of the paper is a random lattice).

This module only describes inputs -- lattice side, species count, circulant
offsets, initial empty fraction, rate parameters, seeds and request streams.
It holds none of the method's arithmetic (both the CUDA path and the oracle
turn these descriptions into digraphs, thresholds and lattices themselves),
so it can serve the tests, the benchmark and the oracle alike.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED0 = 0x5EED0000


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    S: int
    K: tuple            # circulant offsets of the dominance digraph C(S, K)
    p_empty: float      # initial empty-site probability
    interact: float     # mu
    reproduce: float    # sigma
    mobility: float | None = None   # M; exchange rate = 2 M N when given
    exchange: float = 0.0           # used when mobility is None
    n_mcs: int = 100
    log_every: int = 10
    seed: int = SEED0
    extra: dict = field(default_factory=dict)


# The five configurations of the benchmark description (single-lattice ones
# here; the ensemble and request-stream generators are below).
CFG1 = Workload("rps-competition-L64", 64, 3, (1,), 0.0, 1.0, 0.0, None, 0.0, n_mcs=100)
CFG2 = Workload("rpsls-L800-M1e-4", 800, 5, (1, 2), 0.2, 1.0, 1.0, 1e-4, n_mcs=1000)
CFG3 = {M: Workload(f"rps-L3200-M{M:g}", 3200, 3, (1,), 0.25, 1.0, 1.0, M, n_mcs=10000,
                    log_every=10) for M in (1e-5, 1e-4, 1e-3)}


def ensemble(n: int = 1024, seed: int = 1, Ls=(64, 100, 200, 400), Ms=(1e-5, 1e-3),
             max_mcs: int = 10000):
    """Replica specs of the batched-ensemble workload: L uniform over Ls, S
    uniform over {3, 5} (RPS / RPSLS), M log-uniform on Ms, uniform initial
    states over S+1 values, seed SEED0 + index."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        S = int(rng.choice([3, 5]))
        out.append(dict(index=i, L=int(rng.choice(Ls)), S=S, K=(1,) if S == 3 else (1, 2),
                        p_empty=1.0 / (S + 1), interact=1.0, reproduce=1.0,
                        mobility=float(10 ** rng.uniform(np.log10(Ms[0]), np.log10(Ms[1]))),
                        seed=SEED0 + i, max_mcs=max_mcs, stop_at_extinction=True))
    return out


def request_stream(n: int = 10000, seed: int = 2, rate_per_s: float = 1000.0, L_range=(50, 1600),
                   budget_range=(100, 10000), p_stop=0.5):
    """Serving requests: Poisson arrival times, L log-uniform (integer) on
    L_range, S in {3, 5}, MCS budget log-uniform on budget_range, half of
    them stop at extinction; other parameters as the ensemble."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for i in range(n):
        S = int(rng.choice([3, 5]))
        L = int(round(10 ** rng.uniform(np.log10(L_range[0]), np.log10(L_range[1]))))
        out.append(dict(index=i, arrival_s=float(t[i]), L=L, S=S, K=(1,) if S == 3 else (1, 2),
                        p_empty=1.0 / (S + 1), interact=1.0, reproduce=1.0,
                        mobility=float(10 ** rng.uniform(-5, -3)), seed=SEED0 + 100000 + i,
                        max_mcs=int(round(10 ** rng.uniform(np.log10(budget_range[0]),
                                                            np.log10(budget_range[1])))),
                        stop_at_extinction=bool(rng.random() < p_stop)))
    return out


def park_network(alpha: float, beta: float, gamma: float, S: int = 8):
    """(digraph, edge probabilities) of an S-species cyclic network in which
    species a beats a+1, a+2 and a+3 (mod S) with probabilities alpha, beta
    and gamma: the probability structure of Park, Chen and Szolnoki's
    eight-species model.  The paper's figure of their network is missing
    from the text, so this edge set is a stand-in of the same shape."""
    D = np.zeros((S, S), dtype=np.uint8)
    P = np.zeros((S, S))
    for a in range(S):
        for d, p in zip((1, 2, 3), (alpha, beta, gamma)):
            D[a, (a + d) % S] = 1
            P[a, (a + d) % S] = p
    return D, P


def park_ensemble(per_point: int = 64, alphas=(0.2, 0.5, 0.8), betas=(0.2, 0.5, 0.8), gamma: float = 1.0,
                  L: int = 100, seed0: int = SEED0 + 500000):
    """Replica specs of the probabilistic-dominance experiment the paper
    replicates: no mobility, L = 100, 8 species, runs of L^2 MCS (or until
    at most one species is left), per_point seeds at every (alpha, beta)."""
    out = []
    k = 0
    for a in alphas:
        for b in betas:
            D, P = park_network(a, b, gamma)
            for _ in range(per_point):
                out.append(dict(L=L, S=8, digraph=D, dominance_prob=P, rates=(1.0, 1.0, 0.0),
                                seed=seed0 + k, p_empty=0.0, max_mcs=L * L, stop_at_extinction=True,
                                point=(a, b)))
                k += 1
    return out
