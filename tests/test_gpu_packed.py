"""Bit-packed lattices on the GPU (2 or 4 bits per site in device memory):
every launch mode ends bit-identical to the replay oracle, with the counts of
every log point, in both partition geometries, on rectangles and with the
rule variants; the device buffer holds the documented packed layout; host
transfers, validation and size limits behave as with one byte per site."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _decode(raw: np.ndarray, L: int, bits: int) -> np.ndarray:
    """Sites of packed rows (site c at bits [c*bits, (c+1)*bits), little endian)."""
    per = 8 // bits
    b = raw[:, : (L + per - 1) // per]
    fields = [(b >> (bits * e)) & ((1 << bits) - 1) for e in range(per)]
    return np.stack(fields, axis=-1).reshape(raw.shape[0], -1)[:, :L].astype(np.uint8)


@pytest.mark.parametrize("persistent", [1, 3, 5, 0], ids=["persistent", "persistent-flags", "persistent-owner",
                                                          "phase"])
@pytest.mark.parametrize("bits,S,K", [(2, 3, (1,)), (4, 5, (1, 2)), (4, 3, (1,))])
@pytest.mark.parametrize("L,H", [(128, 128), (256, 256), (100, 100), (131, 131), (128, 200), (200, 64), (384, 512)])
def test_packed_parity(L, H, bits, S, K, persistent):
    seed = 7000 + L + 3 * H + bits
    D = O.circulant(S, K)
    X = 2.0 + L / 64
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.2, persistent=persistent, log_every=2, H=H,
                  bits_per_site=bits)
    assert g.update_kernel in ("persistent_kernel", "phase_kernel", "resident_kernel", "persistent_own_kernel",
                               "persistent_gown_kernel")
    o = O.init(L, S, 0.2, seed, H=H)
    assert np.array_equal(g.snapshot(), o)
    m = 0
    for step in (1, 3):
        g.run(step)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, step, mcs_begin=m)
        m += step
        got = g.snapshot()
        assert np.array_equal(got, o), f"after {m} MCS: {int((got != o).sum())} sites differ"
    _, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, X, seed, m, log_every=2)
    assert np.array_equal(log, olog)
    c, _ = g.counts()
    assert np.array_equal(c, O.counts(o, S))


@pytest.mark.parametrize("nbh,reflect", [(8, False), (4, True), (8, True)], ids=["moore", "reflect", "moore-reflect"])
def test_packed_variant_parity(nbh, reflect):
    S, L, H, seed = 3, 72, 130, 91 + nbh
    D = O.circulant(S, (1,))
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.5), seed, p_empty=0.2, log_every=2, neighbourhood=nbh,
                  reflecting_boundary=reflect, H=H, bits_per_site=2)
    g.run(4)
    o, _ = O.replay_run(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, 2.5, seed, 4, neighbourhood=nbh,
                        reflect=reflect)
    assert np.array_equal(g.snapshot(), o)
    _, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed, H=H), D, 1.0, 1.0, 2.5, seed, 4, log_every=2,
                                neighbourhood=nbh, reflect=reflect)
    assert np.array_equal(log, olog)


@pytest.mark.parametrize("bits", [2, 4])
def test_packed_layout_in_device_buffer(bits):
    torch = pytest.importorskip("torch")
    S, L, H = 3, 100, 70
    D = O.circulant(S, (1,))
    nbytes = E.lattice_bytes(L, H, bits)
    assert nbytes == H * E.lattice_pitch(L, bits)
    row_bytes = -(-L * bits // 8)
    assert E.lattice_pitch(L, bits) == -(-row_bytes // 16) * 16
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    g = E.Lattice(L, S, D, (1.0, 1.0, 3.0), 5, p_empty=0.25, device_buffer=buf, H=H, bits_per_site=bits)
    g.run(3)
    g.sync()
    raw = g.as_tensor().cpu().numpy()
    assert raw.shape == (H, E.lattice_pitch(L, bits))
    assert np.array_equal(_decode(raw, L, bits), g.snapshot())
    with pytest.raises(ValueError):
        E.Lattice(L, S, D, (1.0, 1.0, 1.0), 3, device_buffer=buf[:-16], H=H, bits_per_site=bits)


def test_packed_step_host_restore_and_validation():
    S, L, seed = 3, 128, 9
    D = O.circulant(S, (1,))
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25, bits_per_site=2)
    lat = O.init(L, S, 0.25, 123)
    out, counts = g.step_host(lat, 7, 5)
    o, _ = O.replay_run(lat, D, 1.0, 1.0, 2.0, seed, 5, mcs_begin=7)
    assert np.array_equal(out, o)
    assert np.array_equal(counts, O.counts(o, S))
    g.restore(lat, 7)
    g.run(5)
    assert np.array_equal(g.snapshot(), o)
    # S = 2 in 2 bits: the value 3 fits the field but is not a state
    g2 = E.Lattice(L, 2, O.circulant(2, (1,)), (1.0, 1.0, 1.0), 1, bits_per_site=2)
    bad = np.ones((L, L), dtype=np.uint8)
    bad[5, 7] = 3
    with pytest.raises(E.EscgError):
        g2.restore(bad, 0)
    g2.restore(np.ones((L, L), dtype=np.uint8), 0)
    g2.run(2)


def test_packed_bad_options():
    D3, D5 = O.circulant(3, (1,)), O.circulant(5, (1, 2))
    with pytest.raises(E.EscgError, match="S=5"):
        E.Lattice(128, 5, D5, (1.0, 1.0, 1.0), 1, bits_per_site=2)
    with pytest.raises(E.EscgError, match="64"):
        E.Lattice(48, 3, D3, (1.0, 1.0, 1.0), 1, bits_per_site=4)
    with pytest.raises(E.EscgError, match="64"):
        E.Lattice(128, 3, D3, (1.0, 1.0, 1.0), 1, bits_per_site=4, H=40)
    with pytest.raises(E.EscgError, match="bits_per_site"):
        E.Lattice(128, 3, D3, (1.0, 1.0, 1.0), 1, bits_per_site=3)


def test_packed_benchmark_size():
    """L = 3200 with 2 bits per site (2.56 MB instead of 10.24 MB): the
    first MCS matches the oracle and 20 MCS match the one-byte lattice."""
    S, L, seed = 3, 3200, 2508
    D = O.circulant(S, (1,))
    X = 2.0 * 1e-4 * L * L
    a = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, bits_per_site=2)
    b = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25)
    a.run(1)
    o, _ = O.replay_run(O.init(L, S, 0.25, seed), D, 1.0, 1.0, X, seed, 1)
    assert np.array_equal(a.snapshot(), o)
    a.run(19)
    b.run(20)
    assert np.array_equal(a.snapshot(), b.snapshot())
    _, la = a.counts_log()
    _, lb = b.counts_log()
    assert np.array_equal(la, lb)


@pytest.mark.parametrize("bits", [2, 4])
def test_packed_block_owners_L1024(bits):
    """Block owners on a packed lattice (the default at L = 1024): the tiles
    are unpacked once at launch start and packed once at the end; several
    launches, counts at every log point, the device buffer in the packed
    layout."""
    torch = pytest.importorskip("torch")
    S, L, seed, X = 3, 1024, 31 + bits, 6.0
    D = O.circulant(S, (1,))
    buf = torch.zeros(E.lattice_bytes(L, L, bits), dtype=torch.uint8, device="cuda")
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, log_every=3, bits_per_site=bits, device_buffer=buf)
    assert g.update_kernel == "persistent_own_kernel"
    o = O.init(L, S, 0.25, seed)
    g.run(4).run(3)
    o7, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 7)
    assert np.array_equal(g.snapshot(), o7)
    g.sync()
    raw = g.as_tensor().cpu().numpy()
    assert np.array_equal(_decode(raw, L, bits), o7)
    _, log = g.counts_log()
    _, olog, _ = O.run_observed(o, D, 1.0, 1.0, X, seed, 7, log_every=3)
    assert np.array_equal(log, olog)


@pytest.mark.parametrize("bits,S,K", [(2, 3, (1,)), (4, 5, (1, 2))])
@pytest.mark.parametrize("L,ctas", [(128, 8), (384, 6), (1024, 8)])
def test_packed_flag_kernel_128_thread_ctas(L, ctas, bits, S, K):
    """The flag kernel's 128-thread build on a packed lattice (more than 4
    CTAs per SM requested): each thread stages and writes back two pieces of
    the tile, one of them a rim-column site merged into its packed group of
    4; bit-exact after every MCS and at every log point."""
    seed = 9100 + L + bits
    D = O.circulant(S, K)
    X = 2.0 + L / 64
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.2, persistent=3, ctas_per_sm=ctas, log_every=2,
                  bits_per_site=bits)
    assert g.update_kernel == "persistent_kernel"
    o = O.init(L, S, 0.2, seed)
    for m in range(3):
        g.run(1)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=m)
        assert np.array_equal(g.snapshot(), o), m
    g.run(5)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 5, mcs_begin=3)
    assert np.array_equal(g.snapshot(), o)
    _, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed), D, 1.0, 1.0, X, seed, 8, log_every=2)
    assert np.array_equal(log, olog)


@pytest.mark.parametrize("bits", [2, 4])
def test_packed_flag_kernel_128_thread_default_L6400(bits):
    """L = 6400 (2500 blocks per coarse phase) on a packed lattice: the
    default selection runs the flag kernel's 128-thread build; bit-exact
    against the oracle after 2 MCS and equal to the one-byte lattice after 6."""
    L, S, seed = 6400, 3, 6400 + bits
    D = O.circulant(S, (1,))
    X = 2.0 * 1e-4 * L * L
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, bits_per_site=bits)
    assert g.update_kernel == "persistent_kernel"
    g.run(2)
    o, _ = O.replay_run(O.init(L, S, 0.25, seed), D, 1.0, 1.0, X, seed, 2)
    assert np.array_equal(g.snapshot(), o)
    b = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25)
    g.run(4)
    b.run(6)
    assert np.array_equal(g.snapshot(), b.snapshot())
    g.close()
    b.close()
