"""GPU parity of the block-owner kernel on generic partitions
(persistent_gown_kernel: L or H not a multiple of 128, rectangles, the
reflecting boundary, packed lattices): one CTA per 2 x 2 group of blocks
keeps their tiles in shared memory for a whole launch, exchanges only
boundary records and draws the random words of its next visit ahead.
Bit-exact against the schedule-v1 replay oracle after every MCS."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


CASES = [  # (L, H, S, p_empty, X, reflect, n_mcs, log_every)
    (192, None, 3, 0.25, 2.5, False, 6, 3),      # 4 x 4 blocks of 48
    (200, None, 5, 0.2, 8.0, False, 6, 2),       # 50-wide blocks
    (257, None, 3, 0.25, 13.0, False, 5, 3),     # 64 / 65
    (300, None, 5, 0.2, 18.0, False, 5, 10),     # 75-wide: 324 quads, 512-thread CTAs
    (319, None, 3, 0.1, 20.0, False, 4, 1),      # 79 / 80
    (333, None, 4, 0.2, 22.2, False, 5, 4),      # 6 blocks of 55 / 56
    (450, None, 3, 0.25, 40.5, False, 4, 10),
    (800, None, 5, 0.2, 128.0, False, 4, 2),     # the RPSLS workload's partition
    (200, 384, 3, 0.25, 15.4, False, 5, 3),      # rectangles: generic columns, uniform rows
    (333, 130, 5, 0.2, 8.7, False, 5, 2),        # 6 x 2 blocks
    (130, 333, 3, 0.25, 8.7, False, 5, 10),
    (800, 250, 3, 0.25, 40.0, False, 3, 3),
    (200, None, 5, 0.2, 8.0, True, 6, 2),        # reflecting boundary
    (257, 320, 3, 0.25, 16.4, True, 5, 3),
    (384, None, 3, 0.25, 29.5, True, 4, 10),     # uniform partition, reflecting: generic kernel
    (100, None, 3, 0.25, 2.0, False, 6, 3),      # one group (P = 2)
    (100, 64, 5, 0.2, 1.3, True, 6, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}x{c[1] or c[0]}{'-refl' if c[5] else ''}" for c in CASES])
def test_gown_parity_every_mcs(case):
    L, H, S, p_empty, X, reflect, n, log_every = case
    K = (1,) if S != 5 else (1, 2)
    seed = 9100 + L + 7 * (H or L)
    D = O.circulant(S, K)
    g = E.Lattice(L, S, E.circulant(S, K), (1.0, 1.0, X), seed, p_empty=p_empty, persistent=5,
                  log_every=log_every, H=H, reflecting_boundary=reflect)
    assert g.update_kernel == "persistent_gown_kernel"
    o = O.init(L, S, p_empty, seed, H=H)
    for m in range(n):
        g.run(1)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=m, reflect=reflect)
        got = g.snapshot()
        assert np.array_equal(got, o), f"after MCS {m + 1}: {int((got != o).sum())} sites differ"
    # several MCS per launch, launches ending at log points
    g.run(7)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 7, mcs_begin=n, reflect=reflect)
    assert np.array_equal(g.snapshot(), o)
    ms, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, p_empty, seed, H=H), D, 1.0, 1.0, X, seed, n + 7,
                                log_every=log_every, reflect=reflect)
    assert np.array_equal(log, olog)
    c, mcs = g.counts()
    assert mcs == n + 7 and np.array_equal(c, O.counts(o, S))


@pytest.mark.parametrize("L,H,expect", [(200, None, "persistent_gown_kernel"), (333, None, "persistent_gown_kernel"),
                                        (800, None, "persistent_gown_kernel"), (1000, None, "persistent_gown_kernel"),
                                        (2700, None, "persistent_gown_kernel"), (3000, None, "persistent_kernel"),
                                        (100, None, "resident_kernel"), (200, 384, "persistent_gown_kernel"),
                                        (3200, 1600, "persistent_gown_kernel"), (6400, 1600, "persistent_kernel")])
def test_gown_default_choice(L, H, expect):
    """persistent = 1 runs the generic block owners from two groups of 2 x 2
    blocks while the grid needs at most 3 CTAs per SM (2700: 441 groups;
    3200 x 1600: 325); beyond, the flag kernel (3000: 529 groups; 6400 x
    1600: 650); one group (P = 2): whole-lattice residency."""
    g = E.Lattice(L, 3, E.circulant(3, [1]), (1.0, 1.0, 2.0), 9, p_empty=0.25, H=H)
    assert g.update_kernel == expect
    g.close()


def test_gown_cfg2_full_size_launches_of_ten():
    """The RPSLS workload (L = 800, p_empty 0.2, M = 1e-4) in the benchmark's
    launch shape (10 MCS per launch, counts every 10 MCS)."""
    L, S, seed = 800, 5, 0x5EED0002
    X = O.exchange_from_mobility(1e-4, L * L)
    D = O.circulant(S, (1, 2))
    g = E.Lattice(L, S, E.circulant(S, (1, 2)), (1.0, 1.0, X), seed, p_empty=0.2, log_every=10)
    assert g.update_kernel == "persistent_gown_kernel"
    o = O.init(L, S, 0.2, seed)
    for m in (10, 20, 30):
        g.run(10)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 10, mcs_begin=m - 10)
        assert np.array_equal(g.snapshot(), o), m
    ms, log = g.counts_log()
    assert list(ms) == [0, 10, 20, 30] and np.array_equal(log[-1], O.counts(o, S))


def test_gown_stop_at_extinction():
    S, K, L, seed = 3, (1,), 200, 6
    X = O.exchange_from_mobility(3e-4, L * L)
    D = O.circulant(S, K)
    g = E.Lattice(L, S, E.circulant(S, K), (1.0, 1.0, X), seed, p_empty=0.25, log_every=10,
                  stop_at_extinction=True, persistent=5)
    assert g.update_kernel == "persistent_gown_kernel"
    g.run(4000)
    lat, log, mend = O.run_observed(O.init(L, S, 0.25, seed), D, 1.0, 1.0, X, seed, 4000, log_every=10,
                                    stop_at_extinction=True)
    assert g.mcs == mend
    assert np.array_equal(g.snapshot(), lat)
    ms, glog = g.counts_log()
    assert np.array_equal(glog, log) and ms[-1] == mend


@pytest.mark.parametrize("L,bits", [(200, 8), (333, 4), (200, 2)])
def test_gown_restore_other_lattice_at_same_mcs(L, bits):
    """Records left by an earlier run carry epochs the new one may wait for;
    every restore clears them."""
    S, D, seed = 3, E.circulant(3, [1]), 41
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25, persistent=5, bits_per_site=bits)
    assert g.update_kernel == "persistent_gown_kernel"
    for n in (1, 2, 3):
        for k in range(2):
            lat = O.init(L, S, 0.25, 1000 + 10 * n + k)
            g.restore(lat, 0)
            g.run(n)
            ref, _ = O.replay_run(lat, O.circulant(S, [1]), 1.0, 1.0, 2.0, seed, n)
            assert np.array_equal(g.snapshot(), ref), (n, k)


@pytest.mark.parametrize("L,H,bits,S", [(200, None, 2, 3), (333, 200, 4, 5), (257, None, 4, 3),
                                        (300, None, 2, 3)])
def test_gown_packed_parity(L, H, bits, S):
    """Packed rows: tiles unpacked at launch start; at the end the groups a
    block shares with its horizontal neighbour are merged in atomically."""
    K = (1,) if S == 3 else (1, 2)
    seed = 7300 + L + bits
    D = O.circulant(S, K)
    X = 2.0 + L / 64
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.2, persistent=5, log_every=2, H=H,
                  bits_per_site=bits)
    assert g.update_kernel == "persistent_gown_kernel"
    o = O.init(L, S, 0.2, seed, H=H)
    m = 0
    for step in (1, 3, 5):
        g.run(step)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, step, mcs_begin=m)
        m += step
        got = g.snapshot()
        assert np.array_equal(got, o), f"after {m} MCS: {int((got != o).sum())} sites differ"


def test_gown_two_handles_overlapping():
    torch = pytest.importorskip("torch")
    L, S, D, X = 800, 3, E.circulant(3, [1]), 2.0
    hs = [E.Lattice(L, S, D, (1.0, 1.0, X), 100 + i, p_empty=0.25, persistent=5, stream=torch.cuda.Stream())
          for i in range(2)]
    for k in range(6):
        for h in hs:
            h.run(1)
    for h in hs:
        h.sync()
    for i, h in enumerate(hs):
        o, _ = O.replay_run(O.init(L, S, 0.25, 100 + i), O.circulant(S, [1]), 1.0, 1.0, X, 100 + i, 6)
        assert np.array_equal(h.snapshot(), o), i


def test_gown_bounded_wait_times_out_with_status():
    """A block that never publishes its records (host-controlled hook) makes
    its neighbours' bounded waits run out: the kernel returns, escg_sync
    reports ESCG_ETIMEOUT and a restore brings the handle back."""
    L, S = 200, 3
    g = E.Lattice(L, S, E.circulant(S, [1]), (1.0, 1.0, 1.0), 3, p_empty=0.25, persistent=5)
    assert g.update_kernel == "persistent_gown_kernel"
    ref = g.snapshot()
    g.debug_stall_block(5, spin_limit=2000)
    g.run(3)
    with pytest.raises(E.EscgError) as ei:
        g.sync()
    assert ei.value.status == -5
    g.debug_stall_block(-1)
    g.restore(ref, 0)
    g.run(2)
    o, _ = O.replay_run(ref, O.circulant(S, [1]), 1.0, 1.0, 1.0, 3, 2)
    assert np.array_equal(g.snapshot(), o)


@pytest.mark.parametrize("L,per_sm", [(400, 3), (800, 2), (1024, 4), (1024, 8)])
def test_owners_packed_per_sm_concurrent_handles(L, per_sm):
    """Block owners with a packing request (at least per_sm CTAs per SM, the
    other SMs left free): three handles on their own streams, each
    bit-exact against the replay oracle after 5 MCS (generic owners at
    L = 400 and 800, uniform owners at 1024, 128-thread CTAs at 8 per SM)."""
    torch = pytest.importorskip("torch")
    S, X = 3, 3.0
    D = E.circulant(S, [1])
    hs = [E.Lattice(L, S, D, (1.0, 1.0, X), 300 + i, p_empty=0.25, persistent=5, ctas_per_sm=per_sm,
                    stream=torch.cuda.Stream()) for i in range(3)]
    expect = "persistent_own_kernel" if L % 128 == 0 else "persistent_gown_kernel"
    assert all(h.update_kernel == expect for h in hs)
    for h in hs:
        h.run(2)
    for h in hs:
        h.run(3)
    for i, h in enumerate(hs):
        o, _ = O.replay_run(O.init(L, S, 0.25, 300 + i), O.circulant(S, [1]), 1.0, 1.0, X, 300 + i, 5)
        assert np.array_equal(h.snapshot(), o), i
        h.close()
