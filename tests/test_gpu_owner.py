"""GPU parity of the block-owner kernel (persistent = 5): one CTA per 2x2
group of 64x64 blocks keeps their tiles in shared memory for a whole launch
and exchanges only boundary records; bit-exact against the schedule-v1
replay oracle.  The small cases (several launches, log points, restores,
stasis) are in test_gpu_parity.py; here: which lattices it takes, the
benchmark lattice at full size, two handles whose launches overlap, and the
bounded waits."""
import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300 import workloads as W
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("L,H,bits,expect", [(128, None, 8, "persistent_own_kernel"),
                                             (1024, None, 8, "persistent_own_kernel"),
                                             (3200, None, 8, "persistent_own_kernel"),
                                             (100, None, 8, "persistent_gown_kernel"),
                                             (256, 128, 8, "persistent_own_kernel"),
                                             (200, 128, 8, "persistent_gown_kernel"),
                                             (256, None, 2, "persistent_own_kernel"),
                                             (6400, None, 8, "persistent_kernel")])
def test_owner_kernel_choice(L, H, bits, expect):
    """Uniform lattices (squares and rectangles, any bits per site) whose
    (L/128)(H/128) groups the device holds at once run the uniform owner
    kernel, generic partitions (100; 200 x 128) the generic one; 6400 (2500
    groups, more CTAs of 128 threads than 152 SMs can hold) the flag kernel."""
    g = E.Lattice(L, 3, E.circulant(3, [1]), (1.0, 1.0, 1.0), 5, p_empty=0.25, persistent=5, H=H,
                  bits_per_site=bits)
    assert g.update_kernel == expect
    g.close()


def test_owner_cfg3_L3200_full_size():
    """The benchmark lattice (L = 3200, RPS, M = 1e-4) in chunks of 10 MCS
    with counts every 10 MCS, checked after MCS 1, 2 and 10."""
    w = W.CFG3[1e-4]
    X = O.exchange_from_mobility(w.mobility, w.L * w.L) if w.mobility is not None else w.exchange
    D = O.circulant(w.S, w.K)
    g = E.Lattice(w.L, w.S, E.circulant(w.S, w.K), (w.interact, w.reproduce, X), w.seed, p_empty=w.p_empty,
                  log_every=w.log_every, persistent=5)
    assert g.update_kernel == "persistent_own_kernel"
    o = O.init(w.L, w.S, w.p_empty, w.seed)
    m = 0
    for c in (1, 2, 10):
        g.run(c - m)
        o, _ = O.replay_run(o, D, w.interact, w.reproduce, X, w.seed, c - m, mcs_begin=m)
        m = c
        assert np.array_equal(g.snapshot(), o), c
    ms, log = g.counts_log()
    assert list(ms) == [0, 10] and np.array_equal(log[-1], O.counts(o, w.S))


def test_owner_128_thread_ctas_L2048():
    """256 groups on 152 SMs: CTAs of 128 threads, two per SM, each thread
    stepping two quads pairwise; several launches (log points every 2 MCS)."""
    L, S, X, seed = 2048, 5, 40.0, 2048
    D = O.circulant(S, (1, 2))
    g = E.Lattice(L, S, E.circulant(S, (1, 2)), (1.0, 1.0, X), seed, p_empty=0.2, log_every=2, persistent=5)
    assert g.update_kernel == "persistent_own_kernel"
    o = O.init(L, S, 0.2, seed)
    g.run(3)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 3)
    assert np.array_equal(g.snapshot(), o)
    g.run(1)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=3)
    assert np.array_equal(g.snapshot(), o)
    ms, glog = g.counts_log()
    assert list(ms) == [0, 2, 4] and np.array_equal(glog[-1], O.counts(o, S))
    g.run(2)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 2, mcs_begin=4)
    assert np.array_equal(g.snapshot(), o)


@pytest.mark.parametrize("L,n", [(1024, 12), (3200, 3)])
def test_owner_two_handles_overlapping(L, n):
    """Two handles on two streams launched back to back: the cooperative
    launch starts a grid only with all of its CTAs resident (at L = 3200 the
    two grids of 625 CTAs do not fit at once), and both results are exact."""
    torch = pytest.importorskip("torch")
    S, D, X = 3, E.circulant(3, [1]), 2.0
    hs = [E.Lattice(L, S, D, (1.0, 1.0, X), 100 + i, p_empty=0.25, persistent=5, stream=torch.cuda.Stream())
          for i in range(2)]
    for k in range(n):
        for h in hs:
            h.run(1)
    for h in hs:
        h.sync()
    for i, h in enumerate(hs):
        o, _ = O.replay_run(O.init(L, S, 0.25, 100 + i), O.circulant(S, [1]), 1.0, 1.0, X, 100 + i, n)
        assert np.array_equal(h.snapshot(), o), i


def test_owner_bounded_wait_times_out_with_status():
    """A block that never publishes its records (host-controlled hook) makes
    its neighbours' bounded waits run out: the kernel returns, escg_sync
    reports ESCG_ETIMEOUT and a restore brings the handle back.  No hang, no
    fault."""
    L, S = 256, 3
    g = E.Lattice(L, S, E.circulant(S, [1]), (1.0, 1.0, 1.0), 3, p_empty=0.25, persistent=5)
    assert g.update_kernel == "persistent_own_kernel"
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
