"""Probabilistic-edge dominance (Park, Chen and Szolnoki's model as the
paper's section "Park, Chen, Szolnoki" describes it) on the GPU: every launch
mode of the single-lattice path, the batched ensemble and the server end
bit-identical to the replay oracle with the same edge probabilities."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _park8(alpha, beta, gamma):
    """8-species cyclic network, each species beating the next three with
    edge probabilities alpha, beta, gamma (a stand-in for the paper's
    missing figure: the structure of the probabilities, not its edges)."""
    S = 8
    D = O.circulant(S, (1, 2, 3))
    P = np.zeros((S, S))
    for a in range(S):
        for d, p in zip((1, 2, 3), (alpha, beta, gamma)):
            P[a, (a + d) % S] = p
    return D, P


@pytest.mark.parametrize("persistent", [1, 3, 2, 0], ids=["persistent", "persistent-flags", "persistent-tma", "phase"])
@pytest.mark.parametrize("L,n", [(100, 6), (128, 5), (256, 4), (131, 4)])
def test_single_lattice_parity(L, n, persistent):
    D, P = _park8(0.3, 0.6, 1.0)
    S, seed = 8, 9000 + L
    g = E.Lattice(L, S, D, (1.0, 0.0, 0.0), seed, p_empty=0.0, persistent=persistent, log_every=2,
                  dominance_prob=P)
    o = O.init(L, S, 0.0, seed)
    m = 0
    for step in (1, 2, n - 3):
        g.run(step)
        o, _ = O.replay_run(o, D, 1.0, 0.0, 0.0, seed, step, mcs_begin=m, prob=P)
        m += step
        got = g.snapshot()
        assert np.array_equal(got, o), f"after {m} MCS: {int((got != o).sum())} sites differ"
    c, mcs = g.counts()
    assert mcs == m and np.array_equal(c, O.counts(o, S))


def test_mixed_rates_and_zero_edges():
    """Mobility and reproduction together with probabilistic edges, some of
    them impossible (p = 0) -- the same as removing those edges."""
    S, L, seed = 5, 192, 31
    D = O.circulant(S, (1, 2))
    P = np.where(D > 0, 0.45, 0.0)
    P[0, 1] = 0.0
    P[3, 0] = 1.0
    g = E.Lattice(L, S, D, (1.0, 1.0, 3.0), seed, p_empty=0.2, dominance_prob=P)
    g.run(3)
    o, _ = O.replay_run(O.init(L, S, 0.2, seed), D, 1.0, 1.0, 3.0, seed, 3, prob=P)
    assert np.array_equal(g.snapshot(), o)


def test_probability_one_matches_deterministic_lattice():
    S, L, seed = 3, 256, 5
    D = O.circulant(S, (1,))
    a = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25, dominance_prob=np.where(D > 0, 1.0, 0.0))
    b = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25)
    a.run(4)
    b.run(4)
    assert np.array_equal(a.snapshot(), b.snapshot())


def test_batch_and_server_parity():
    D, P = _park8(0.5, 0.8, 1.0)
    specs = []
    for i, L in enumerate([64, 100, 150, 200]):
        specs.append(dict(L=L, S=8, digraph=D, rates=(1.0, 0.0, 0.0), seed=777 + i, p_empty=0.0,
                          max_mcs=12 + 3 * i, stop_at_extinction=False,
                          dominance_prob=P if i % 2 == 0 else np.where(D > 0, 0.25, 0.0)))
    b = E.Batch(specs, log_every=4)
    b.run()
    srv = E.Server(arena_bytes=64 << 20, max_slots=8, log_every=4, keep_lattice=True)
    ids = [srv.submit(sp) for sp in specs]
    while srv.stats()[0] or srv.stats()[1]:
        srv.step()
    for i, sp in enumerate(specs):
        o, _ = O.replay_run(O.init(sp["L"], 8, 0.0, sp["seed"]), D, 1.0, 0.0, 0.0, sp["seed"],
                            sp["max_mcs"], prob=sp["dominance_prob"])
        assert np.array_equal(b.snapshot(i), o), i
        mcs, _, _, lat = srv.result(ids[i], lattice=True)
        assert mcs == sp["max_mcs"] and np.array_equal(lat, o), i


def test_invalid_probability_is_rejected():
    D = O.circulant(3, (1,))
    with pytest.raises(E.EscgError):
        E.Lattice(64, 3, D, (1.0, 1.0, 1.0), 1, dominance_prob=np.full((3, 3), 1.5))
