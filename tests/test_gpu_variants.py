"""Rule variants on the GPU (the paper's --neighbourhood 8 and reflecting
--flux false): every launch mode of the single-lattice path ends
bit-identical to the replay oracle, with the counts of every log point."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("persistent", [1, 3, 2, 5, 0],
                         ids=["persistent", "persistent-flags", "persistent-tma", "persistent-owner", "phase"])
@pytest.mark.parametrize("nbh,reflect", [(8, False), (4, True), (8, True)], ids=["moore", "reflect", "moore-reflect"])
@pytest.mark.parametrize("L", [64, 128, 131, 256])
def test_variant_parity(L, nbh, reflect, persistent):
    S, K, seed = 5, (1, 2), 4000 + L + 17 * nbh + int(reflect)
    D = O.circulant(S, K)
    X = 2.0 + L / 64
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.2, persistent=persistent, log_every=2,
                  neighbourhood=nbh, reflecting_boundary=reflect)
    o = O.init(L, S, 0.2, seed)
    m = 0
    for step in (1, 3):
        g.run(step)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, step, mcs_begin=m, neighbourhood=nbh, reflect=reflect)
        m += step
        got = g.snapshot()
        assert np.array_equal(got, o), f"after {m} MCS: {int((got != o).sum())} sites differ"
    ms, log = g.counts_log()
    lat, olog, _ = O.run_observed(O.init(L, S, 0.2, seed), D, 1.0, 1.0, X, seed, m, log_every=2,
                                  neighbourhood=nbh, reflect=reflect)
    assert np.array_equal(log, olog)


def test_variant_stop_at_extinction():
    S, L, seed = 3, 48, 77
    D = O.circulant(S, (1,))
    g = E.Lattice(L, S, D, (1.0, 1.0, 0.3), seed, p_empty=0.25, log_every=5, stop_at_extinction=True,
                  neighbourhood=8, reflecting_boundary=True)
    g.run(400)
    lat, log, mend = O.run_observed(O.init(L, S, 0.25, seed), D, 1.0, 1.0, 0.3, seed, 400, log_every=5,
                                    stop_at_extinction=True, neighbourhood=8, reflect=True)
    assert g.mcs == mend
    assert np.array_equal(g.snapshot(), lat)


def test_bad_variant_is_rejected():
    D = O.circulant(3, (1,))
    with pytest.raises(E.EscgError):
        E.Lattice(64, 3, D, (1.0, 1.0, 1.0), 1, neighbourhood=6)


@pytest.mark.parametrize("nbh,reflect", [(8, False), (4, True), (8, True)], ids=["moore", "reflect", "moore-reflect"])
def test_uniform_variant_visit_full_size(nbh, reflect):
    """The benchmark lattice (L = 3200, 64 x 64 blocks) under the rule
    variants runs the flag kernel's uniform variant visit (the Moore step
    from a byte-permute offset table, the mirror only in blocks on the
    lattice edge); bit-exact against the replay oracle after MCS 1 and 2."""
    L, S, seed = 3200, 3, 3200 + nbh + int(reflect)
    D = O.circulant(S, (1,))
    X = 2.0 * 1e-4 * L * L
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, persistent=3, neighbourhood=nbh,
                  reflecting_boundary=reflect)
    o = O.init(L, S, 0.25, seed)
    for m in range(2):
        g.run(1)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=m, neighbourhood=nbh, reflect=reflect)
        got = g.snapshot()
        assert np.array_equal(got, o), f"after MCS {m + 1}: {int((got != o).sum())} sites differ"


@pytest.mark.parametrize("nbh,reflect", [(4, False), (8, True)], ids=["vonneumann", "moore-reflect"])
def test_deep_generic_visit_full_size(nbh, reflect):
    """L = 4800 (a generic partition of 38 x 38 groups, too many for the block
    owners; 1444 blocks per coarse phase, over two waves of flag-kernel CTAs):
    the flag kernel's generic visit, bit-exact against the replay oracle after
    MCS 1 and 2."""
    L, S, seed = 4800, 3, 4800 + nbh
    D = O.circulant(S, (1,))
    X = 2.0 * 1e-4 * L * L
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, neighbourhood=nbh, reflecting_boundary=reflect)
    assert g.update_kernel == "persistent_kernel"
    o = O.init(L, S, 0.25, seed)
    for m in range(2):
        g.run(1)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=m, neighbourhood=nbh, reflect=reflect)
        got = g.snapshot()
        assert np.array_equal(got, o), f"after MCS {m + 1}: {int((got != o).sum())} sites differ"
