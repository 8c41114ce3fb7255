"""Rectangular L x H lattices on the GPU (the paper's --length and --height):
every launch mode of the single-lattice path ends bit-identical to the
replay oracle, with the counts of every log point, in both geometries of the
partition (uniform 64 x 64 blocks along both axes, and generic ones), with
the rule variants, through the host-buffer call, and at a large size by
properties."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu

MODES = [1, 3, 2, 5, 0]
MODE_IDS = ["persistent", "persistent-flags", "persistent-tma", "persistent-owner", "phase"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


@pytest.mark.parametrize("persistent", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("L,H", [(40, 24), (24, 57), (131, 70), (256, 128), (128, 384), (64, 200), (384, 768),
                                 (1024, 256)])
def test_rect_parity(L, H, persistent):
    S, K, seed = 5, (1, 2), 5000 + L + 3 * H
    D = O.circulant(S, K)
    X = 2.0 + L / 64
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.2, persistent=persistent, log_every=2, H=H)
    o = O.init(L, S, 0.2, seed, H=H)
    assert np.array_equal(g.snapshot(), o)
    m = 0
    for step in (1, 3):
        g.run(step)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, step, mcs_begin=m)
        m += step
        got = g.snapshot()
        assert got.shape == (H, L)
        assert np.array_equal(got, o), f"after {m} MCS: {int((got != o).sum())} sites differ"
    ms, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, X, seed, m, log_every=2)
    assert np.array_equal(log, olog)
    assert list(ms) == [0, 2, 4]


@pytest.mark.parametrize("persistent", [1, 0], ids=["persistent", "phase"])
@pytest.mark.parametrize("nbh,reflect", [(8, False), (4, True), (8, True)], ids=["moore", "reflect", "moore-reflect"])
def test_rect_variant_parity(nbh, reflect, persistent):
    S, L, H, seed = 5, 72, 130, 61 + nbh
    D = O.circulant(S, (1, 2))
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.5), seed, p_empty=0.2, persistent=persistent, log_every=2,
                  neighbourhood=nbh, reflecting_boundary=reflect, H=H)
    g.run(4)
    o, _ = O.replay_run(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, 2.5, seed, 4, neighbourhood=nbh,
                        reflect=reflect)
    assert np.array_equal(g.snapshot(), o)
    _, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, 2.5, seed, 4, log_every=2,
                                neighbourhood=nbh, reflect=reflect)
    assert np.array_equal(log, olog)


def test_rect_step_host_and_restore():
    S, L, H, seed = 3, 96, 40, 9
    D = O.circulant(S, (1,))
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25, H=H)
    lat = O.init(L, S, 0.25, 123, H=H)
    out, counts = g.step_host(lat, 7, 5)
    o, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, seed, 5, mcs_begin=7)
    assert np.array_equal(out, o)
    assert np.array_equal(counts, O.counts(o, S))
    g.restore(lat, 7)
    g.run(5)
    assert np.array_equal(g.snapshot(), o)
    with pytest.raises(ValueError):
        g.restore(np.zeros((L, L), dtype=np.uint8), 0)


def test_rect_device_buffer_and_bad_height():
    torch = pytest.importorskip("torch")
    S, L, H = 3, 64, 24
    D = O.circulant(S, (1,))
    assert E.lattice_bytes(L, H) == H * E.lattice_pitch(L)
    buf = torch.zeros(E.lattice_bytes(L, H), dtype=torch.uint8, device="cuda")
    g = E.Lattice(L, S, D, (1.0, 1.0, 1.0), 3, p_empty=0.1, device_buffer=buf, H=H)
    torch.cuda.synchronize()
    assert np.array_equal(g.as_tensor()[:, :L].cpu().numpy(), O.init(L, S, 0.1, 3, H=H))
    with pytest.raises(ValueError):
        E.Lattice(L, S, D, (1.0, 1.0, 1.0), 3, device_buffer=buf[:-1], H=H)
    # a buffer that is not 16-byte aligned is refused before any launch
    big = torch.zeros(E.lattice_bytes(L, H) + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(E.EscgError, match="aligned"):
        E.Lattice(L, S, D, (1.0, 1.0, 1.0), 3, device_buffer=big[1:], H=H)
    for bad in (7, 16385):
        with pytest.raises(E.EscgError):
            E.Lattice(L, S, D, (1.0, 1.0, 1.0), 3, H=bad)


def test_rect_large_properties():
    """3200 x 1600 (a strip of the 3200 x 3200 benchmark lattice): the default
    kernel (generic block owners: 1600 is not a multiple of 128) matches the
    oracle's replay after the first MCS, it and one launch per coarse phase
    agree bit for bit after 20 MCS, and the logged counts sum to N = L*H."""
    S, L, H, seed = 3, 3200, 1600, 2508
    D = O.circulant(S, (1,))
    X = 2.0 * 1e-4 * L * H
    a = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, persistent=1, H=H)
    b = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, persistent=0, H=H)
    assert a.update_kernel == "persistent_gown_kernel"
    a.run(1)
    o, _ = O.replay_run(O.init(L, S, 0.25, seed, H=H), D, 1.0, 1.0, X, seed, 1)
    assert np.array_equal(a.snapshot(), o)
    a.run(19)
    b.run(20)
    assert np.array_equal(a.snapshot(), b.snapshot())
    _, log = a.counts_log()
    assert (log.sum(axis=1) == L * H).all()


@pytest.mark.parametrize("L,H,expect", [(384, 768, "persistent_own_kernel"), (1024, 256, "persistent_own_kernel"),
                                        (256, 128, "persistent_kernel"), (200, 384, "persistent_gown_kernel")])
def test_rect_default_kernel(L, H, expect):
    """persistent = 1 runs block owners on uniform rectangles from 3 x 3
    groups of 2 x 2 blocks (384 x 768: 3 x 6 groups; 1024 x 256: 8 x 2),
    the flag kernel on smaller ones, the generic block owners on generic
    ones (200 x 384: 2 x 3 groups)."""
    g = E.Lattice(L, 3, E.circulant(3, [1]), (1.0, 1.0, 2.0), 9, p_empty=0.25, H=H)
    assert g.update_kernel == expect
    g.run(4)
    o, _ = O.replay_run(O.init(L, 3, 0.25, 9, H=H), O.circulant(3, [1]), 1.0, 1.0, 2.0, 9, 4)
    assert np.array_equal(g.snapshot(), o)
