"""The autotuner (escg_options.autotune): the first handle of a lattice size
and rule times every distinct launch mode and CTA count on a copy of its
initial lattice and keeps the fastest; later handles of that key reuse the
cached choice.  Whatever it picks, the lattice is the replay oracle's, and
the handle starts at MCS 0 from its initial lattice as if just created."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu

MODES = {1, 2, 3, 4, 5, 6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("L,H,S,bits,reflect", [(128, None, 3, 8, False), (200, None, 5, 8, False),
                                                (800, None, 5, 8, False), (1024, None, 3, 8, False),
                                                (3200, None, 3, 8, False), (256, 128, 3, 8, False),
                                                (384, None, 3, 2, False), (333, None, 3, 8, True)])
def test_autotuned_handle_matches_oracle_and_caches(L, H, S, bits, reflect):
    K = (1,) if S == 3 else (1, 2)
    D = O.circulant(S, K)
    X = 2.0 * 1e-4 * L * (H or L)
    seed = 777 + L
    g = E.Lattice(L, S, E.circulant(S, K), (1.0, 1.0, X), seed, p_empty=0.2, log_every=5, H=H,
                  bits_per_site=bits, reflecting_boundary=reflect, autotune=True)
    mode, ctas, ms, n = g.autotune_result
    assert mode in MODES and ctas in (0, 2, 3) and ms > 0
    assert g.mcs == 0
    o = O.init(L, S, 0.2, seed, H=H)
    assert np.array_equal(g.snapshot(), o), "the tuning runs must leave the initial lattice"
    ms_log, _ = g.counts_log()
    assert list(ms_log) == [0]
    g.run(7)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 7, reflect=reflect)
    assert np.array_equal(g.snapshot(), o)
    # a second handle of the same key takes the cached choice (nothing timed)
    h = E.Lattice(L, S, E.circulant(S, K), (1.0, 1.0, X), seed + 1, p_empty=0.2, H=H, bits_per_site=bits,
                  reflecting_boundary=reflect, autotune=True)
    assert h.autotune_result[:2] == (mode, ctas) and h.autotune_result[3] == 0
    assert h.update_kernel == g.update_kernel
    if n:   # this process tuned the key with g
        assert n >= 2
    g.close()
    h.close()


def test_autotune_result_needs_autotune():
    g = E.Lattice(64, 3, E.circulant(3, [1]), (1.0, 1.0, 1.0), 1)
    with pytest.raises(E.EscgError):
        g.autotune_result
    g.close()


def test_batch_tuner_picks_a_staging_and_keeps_results():
    """The batch engine's first chunks time its chunk kernel at three CTA sizes,
    TMA-staged and plain; the results equal single-lattice runs."""
    specs = []
    for i, L in enumerate((64, 100, 200, 130)):
        S = 3 if i % 2 == 0 else 5
        specs.append(dict(L=L, S=S, digraph=E.circulant(S, (1,) if S == 3 else (1, 2)),
                          rates=(1.0, 1.0, 2.0 * 1e-4 * L * L), seed=40 + i, p_empty=0.2, max_mcs=120,
                          stop_at_extinction=False))
    b = E.Batch(specs, log_every=10, threads=0)
    b.run()
    assert b.threads in (64, 128, 256) and b.uses_tma in (True, False)
    mcs, _, _ = b.status()
    for i, sp in enumerate(specs):
        g = E.Lattice(sp["L"], sp["S"], sp["digraph"], sp["rates"], sp["seed"], p_empty=sp["p_empty"], log_every=10)
        g.run(sp["max_mcs"])
        assert mcs[i] == 120 and np.array_equal(b.snapshot(i), g.snapshot()), i
        g.close()
    b.close()
