"""Batched ensembles on the GPU: every replica of a batch (uneven L, mixed
S, rates, seeds, budgets, stop-at-extinction) ends bit-identical to the same
replica run alone through the single-lattice C ABI and to the replay oracle;
results do not depend on the CTA size, on graph capture or on how the run is
split into calls."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _specs(n=24, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        S = int(rng.choice([3, 5]))
        L = int(rng.choice([8, 13, 31, 64, 100, 131, 200]))
        M = float(10 ** rng.uniform(-3.5, -1.0))
        X = 2 * M * L * L
        out.append(dict(L=L, S=S, K=(1,) if S == 3 else (1, 2),
                        digraph=O.circulant(S, (1,) if S == 3 else (1, 2)),
                        rates=(1.0, 1.0, X), seed=0x5EED0000 + 1000 * seed + i,
                        p_empty=1.0 / (S + 1), max_mcs=int(rng.integers(5, 120)),
                        stop_at_extinction=bool(rng.random() < 0.6)))
    return out


def _alone(sp, log_every):
    g = E.Lattice(sp["L"], sp["S"], E.circulant(sp["S"], sp["K"]), sp["rates"], sp["seed"],
                  p_empty=sp["p_empty"], log_every=log_every,
                  stop_at_extinction=sp["stop_at_extinction"])
    g.run(sp["max_mcs"])
    return g


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_batch_matches_single_runs(threads):
    specs = _specs()
    b = E.Batch(specs, log_every=10, threads=threads)
    b.run()
    mcs, ext, cnt = b.status()
    assert b.active == 0
    for i, sp in enumerate(specs):
        g = _alone(sp, 10)
        assert mcs[i] == g.mcs, i
        assert np.array_equal(b.snapshot(i), g.snapshot()), i
        ms, log = g.counts_log()
        assert np.array_equal(cnt[i, :sp["S"] + 1], log[-1]), i
        assert bool(ext[i]) == (sp["stop_at_extinction"] and (log[-1][1:] > 0).sum() <= 1), i


def test_batch_matches_oracle_and_extinction_flags():
    specs = _specs(n=12, seed=11)
    b = E.Batch(specs, log_every=5, threads=0)
    b.run()
    mcs, ext, cnt = b.status()
    assert b.threads in (64, 128, 256)
    for i, sp in enumerate(specs):
        o = O.init(sp["L"], sp["S"], sp["p_empty"], sp["seed"])
        lat, log, mend = O.run_observed(o, sp["digraph"], *sp["rates"], sp["seed"], sp["max_mcs"],
                                        log_every=5, stop_at_extinction=sp["stop_at_extinction"])
        assert mcs[i] == mend, i
        assert np.array_equal(b.snapshot(i), lat), i
        assert np.array_equal(cnt[i, :sp["S"] + 1], log[-1]), i
        assert bool(ext[i]) == (sp["stop_at_extinction"] and (log[-1][1:] > 0).sum() <= 1), i


def test_batch_graph_and_split_runs_are_invisible():
    specs = _specs(n=16, seed=3)
    a = E.Batch(specs, log_every=10, threads=128, use_graph=True)
    a.run()
    c = E.Batch(specs, log_every=10, threads=128, use_graph=False)
    c.run(30).run(40).run()
    ma, ea, ca = a.status()
    mc, ec, cc = c.status()
    assert np.array_equal(ma, mc) and np.array_equal(ea, ec) and np.array_equal(ca, cc)
    for i in range(len(specs)):
        assert np.array_equal(a.snapshot(i), c.snapshot(i))


def test_batch_single_replica_and_immediate_extinction():
    D = O.circulant(3, [1])
    mono = dict(L=16, S=3, K=(1,), digraph=D, rates=(1.0, 1.0, 1.0), seed=5, p_empty=1.0,
                max_mcs=50, stop_at_extinction=True)   # all empty: extinct at MCS 0
    b = E.Batch([mono], log_every=10, threads=64)
    b.run()
    mcs, ext, cnt = b.status()
    assert mcs[0] == 0 and ext[0] and cnt[0, 0] == 256


def test_batch_resident_classes_match_chunk_kernel():
    """Replicas of every whole-lattice residency class (L 8..131, 200,
    448) next to ones that stay in the block-by-block chunk kernel (L 600):
    the same lattices, MCS numbers, counts and extinction flags with
    residency on and off, and the oracle for a sample."""
    specs = _specs(n=10, seed=21)
    rng = np.random.default_rng(5)
    for i, L in enumerate([448, 600, 448, 600]):
        S = 3
        specs.append(dict(L=L, S=S, K=(1,), digraph=O.circulant(S, (1,)), rates=(1.0, 1.0, 2e-4 * L * L),
                          seed=0x5EED7000 + i, p_empty=0.25, max_mcs=int(rng.integers(12, 40)),
                          stop_at_extinction=False))
    a = E.Batch(specs, log_every=10, threads=128, resident=True)
    a.run()
    c = E.Batch(specs, log_every=10, threads=128, resident=False)
    c.run()
    ma, ea, ca = a.status()
    mc, ec, cc = c.status()
    assert np.array_equal(ma, mc) and np.array_equal(ea, ec) and np.array_equal(ca, cc)
    for i in range(len(specs)):
        assert np.array_equal(a.snapshot(i), c.snapshot(i)), i
    for i in (0, 3, len(specs) - 4):
        sp = specs[i]
        o = O.init(sp["L"], sp["S"], sp["p_empty"], sp["seed"])
        lat, log, mend = O.run_observed(o, sp["digraph"], *sp["rates"], sp["seed"], sp["max_mcs"],
                                        log_every=10, stop_at_extinction=sp["stop_at_extinction"])
        assert ma[i] == mend and np.array_equal(a.snapshot(i), lat), i
