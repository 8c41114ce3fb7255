"""Whole-lattice residency on the GPU (persistent = 4: the lattice stays in
one CTA's shared memory for every coarse phase of a launch): bit-identical to
the replay oracle, with the counts of every log point, in both partition
geometries, on rectangles, with the rule variants and packed storage; larger
lattices fall back to the flag kernel."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("L,H", [(8, 8), (13, 40), (64, 64), (100, 100), (128, 128), (131, 131), (200, 200),
                                 (256, 256), (128, 320), (448, 448)])
@pytest.mark.parametrize("S,K", [(3, (1,)), (5, (1, 2))])
def test_resident_parity(L, H, S, K):
    seed = 9000 + L + 7 * H + S
    D = O.circulant(S, K)
    X = 2.0 + L / 64
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.2, persistent=4, log_every=2, H=H)
    assert g.update_kernel == "resident_kernel"
    o = O.init(L, S, 0.2, seed, H=H)
    m = 0
    for step in (1, 4):
        g.run(step)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, step, mcs_begin=m)
        m += step
        got = g.snapshot()
        assert np.array_equal(got, o), f"after {m} MCS: {int((got != o).sum())} sites differ"
    ms, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, X, seed, m, log_every=2)
    assert np.array_equal(log, olog)
    assert list(ms) == [0, 2, 4]
    assert g.mcs == m


@pytest.mark.parametrize("nbh,reflect", [(8, False), (4, True), (8, True)], ids=["moore", "reflect", "moore-reflect"])
@pytest.mark.parametrize("L,H", [(72, 130), (128, 128), (9, 11)])
def test_resident_variant_parity(L, H, nbh, reflect):
    S, seed = 5, 301 + L + nbh
    D = O.circulant(S, (1, 2))
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.5), seed, p_empty=0.2, persistent=4, log_every=2, neighbourhood=nbh,
                  reflecting_boundary=reflect, H=H)
    g.run(5)
    o, _ = O.replay_run(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, 2.5, seed, 5, neighbourhood=nbh,
                        reflect=reflect)
    assert np.array_equal(g.snapshot(), o)
    _, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, 2.5, seed, 5, log_every=2,
                                neighbourhood=nbh, reflect=reflect)
    assert np.array_equal(log, olog)


@pytest.mark.parametrize("bits", [2, 4])
def test_resident_packed_and_probabilities(bits):
    S, L, seed = 3, 160, 44
    D = O.circulant(S, (1,))
    P = np.zeros((S, S))
    P[D.astype(bool)] = 0.6
    g = E.Lattice(L, S, D, (1.0, 1.0, 1.5), seed, p_empty=0.25, persistent=4, bits_per_site=bits,
                  dominance_prob=P)
    g.run(6)
    o, _ = O.replay_run(O.init(L, S, 0.25, seed), D, 1.0, 1.0, 1.5, seed, 6, prob=P)
    assert np.array_equal(g.snapshot(), o)


def test_resident_stop_at_extinction_and_step_host():
    S, L, seed = 3, 48, 77
    D = O.circulant(S, (1,))
    g = E.Lattice(L, S, D, (1.0, 1.0, 0.3), seed, p_empty=0.25, log_every=5, stop_at_extinction=True,
                  persistent=4)
    g.run(2000)
    lat, log, mend = O.run_observed(O.init(L, S, 0.25, seed), D, 1.0, 1.0, 0.3, seed, 2000, log_every=5,
                                    stop_at_extinction=True)
    assert g.mcs == mend
    assert np.array_equal(g.snapshot(), lat)
    _, glog = g.counts_log()
    assert np.array_equal(glog, log)
    h = E.Lattice(100, S, D, (1.0, 1.0, 2.0), 5, p_empty=0.2, persistent=4)
    lat0 = O.init(100, S, 0.2, 99)
    out, counts = h.step_host(lat0, 3, 7)
    o, _ = O.replay_run(lat0, D, 1.0, 1.0, 2.0, 5, 7, mcs_begin=3)
    assert np.array_equal(out, o)
    assert np.array_equal(counts, O.counts(o, S))


def test_resident_fallback_for_large_lattices():
    D = O.circulant(3, (1,))
    g = E.Lattice(800, 3, D, (1.0, 1.0, 2.0), 1, persistent=4)
    assert g.update_kernel == "persistent_kernel"
    g.run(2)
    o, _ = O.replay_run(O.init(800, 3, 0.0, 1), D, 1.0, 1.0, 2.0, 1, 2)
    assert np.array_equal(g.snapshot(), o)


@pytest.mark.parametrize("L,H,expect", [(100, 100, "resident_kernel"), (64, 150, "resident_kernel"),
                                        (128, 128, "persistent_ll_kernel"), (384, 384, "persistent_own_kernel"),
                                        (200, 200, "persistent_gown_kernel"),
                                        (2048, 2048, "persistent_own_kernel"), (2816, 2816, "persistent_kernel"),
                                        (256, 128, "persistent_kernel")])
def test_default_kernel_choice(L, H, expect):
    """persistent = 1 picks residency for generic 2 x 2-block partitions,
    the generic block owners for larger generic ones (200: 2 x 2 groups),
    for uniform square ones the mailbox kernel below 3 x 3 groups of blocks
    (128), block owners up to 3 owner CTAs per SM (384; 2048: 256 groups),
    the flag kernel beyond (2816: 484 groups) and for small rectangles."""
    D = O.circulant(3, (1,))
    g = E.Lattice(L, 3, D, (1.0, 1.0, 2.0), 11, p_empty=0.2, H=H)
    assert g.update_kernel == expect
    g.run(3)
    o, _ = O.replay_run(O.init(L, 3, 0.2, 11, H=H), D, 1.0, 1.0, 2.0, 11, 3)
    assert np.array_equal(g.snapshot(), o)
