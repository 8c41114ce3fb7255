"""GPU parity: the CUDA path (through the C ABI) against the schedule-v1
replay oracle, bit-exact (integer lattice work), after every MCS.

Covers small and ragged lattices (odd L, non-uniform partitions, several
tiles), the three benchmark lattices at their full sizes in the launch
configuration the benchmark times (persistent kernel, default grid), both
launch modes, counts and the count log, stasis, exact resume, the
end-to-end host call and torch memory/stream interop.
"""
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


def _x(L, mobility, exchange):
    return O.exchange_from_mobility(mobility, L * L) if mobility is not None else exchange


def _pair(L, S, K, p_empty, I, P, X, seed, **kw):
    D = O.circulant(S, K)
    g = E.Lattice(L, S, E.circulant(S, K), (I, P, X), seed, p_empty=p_empty, **kw)
    o = O.init(L, S, p_empty, seed)
    return g, o, D


@pytest.mark.parametrize("L,S,p_empty,seed", [(8, 3, 0.0, 1), (13, 5, 0.2, 2), (64, 3, 0.25, 3),
                                              (100, 5, 1 / 6, 4), (333, 7, 0.5, 5), (800, 5, 0.2, 6),
                                              (3200, 3, 0.25, W.SEED0), (16, 3, 1.0, 7)])
def test_init_matches_oracle(L, S, p_empty, seed):
    g, o, _ = _pair(L, S, [1], p_empty, 1.0, 1.0, 1.0, seed)
    assert np.array_equal(g.snapshot(), o)
    c, m = g.counts()
    assert m == 0 and np.array_equal(c, O.counts(o, S))


SMALL = [  # (L, S, K, p_empty, I, P, X, n_mcs)
    (8, 3, (1,), 0.25, 1.0, 1.0, 1.0, 12),
    (9, 3, (1,), 0.25, 1.0, 1.0, 0.3, 10),
    (12, 5, (1, 2), 0.2, 1.0, 1.0, 2.0, 10),
    (13, 3, (1,), 0.0, 1.0, 0.0, 0.0, 10),
    (31, 5, (1, 2), 1 / 6, 0.5, 1.5, 4.0, 8),
    (50, 3, (1,), 0.25, 1.0, 1.0, 0.5, 8),
    (64, 3, (1,), 0.25, 1.0, 1.0, 0.8192, 8),
    (77, 5, (1, 2), 0.2, 1.0, 1.0, 11.86, 6),
    (100, 3, (1,), 0.25, 1.0, 1.0, 2.0, 6),
    (131, 4, (1,), 0.1, 1.0, 2.0, 1.0, 5),
    (191, 3, (1,), 0.25, 1.0, 1.0, 7.3, 4),
    (200, 5, (1, 2), 0.2, 1.0, 1.0, 8.0, 4),
    (257, 3, (1,), 0.25, 0.0, 0.0, 1.0, 3),
    (128, 3, (1,), 0.25, 1.0, 1.0, 3.3, 5),      # uniform 64x64 blocks, P = 2
    (256, 5, (1, 2), 0.2, 1.0, 1.0, 13.1, 4),    # uniform, P = 4
    (384, 3, (1,), 0.25, 1.0, 1.0, 29.5, 3),     # uniform, P = 6
]


@pytest.mark.parametrize("persistent", [1, 3, 2, 5, 6, 0],
                         ids=["persistent", "persistent-flags", "persistent-tma", "persistent-owner",
                              "persistent-mailbox", "phase"])
@pytest.mark.parametrize("case", SMALL, ids=[f"L{c[0]}" for c in SMALL])
def test_replay_parity_every_mcs(case, persistent):
    L, S, K, p_empty, I, P, X, n = case
    seed = 1000 + L
    g, o, D = _pair(L, S, K, p_empty, I, P, X, seed, persistent=persistent, log_every=3)
    for m in range(n):
        g.run(1)
        o, att = O.replay_run(o, D, I, P, X, seed, 1, mcs_begin=m)
        assert att == L * L
        got = g.snapshot()
        assert np.array_equal(got, o), f"L={L} mismatch after MCS {m + 1}: " \
                                       f"{int((got != o).sum())} sites differ"
    c, mcs = g.counts()
    assert mcs == n and np.array_equal(c, O.counts(o, S))


@pytest.mark.parametrize("persistent", [1, 3, 5, 6],
                         ids=["persistent", "persistent-flags", "persistent-owner", "persistent-mailbox"])
@pytest.mark.parametrize("L,S,X,n,log_every", [(128, 3, 3.3, 7, 10), (256, 5, 13.1, 5, 2), (384, 3, 29.5, 4, 3),
                                               (640, 4, 50.0, 3, 10)])
def test_many_mcs_per_launch(L, S, X, n, log_every, persistent):
    """Several MCS in one launch (and several launches per run when log
    points end them): the coarse colour order changes every MCS, so a
    block's neighbours may have visited before or after its own previous
    visit -- exactly what the boundary records must get right."""
    seed = 4242 + L
    K = (1,) if S == 3 else (1, 2)
    g, o, D = _pair(L, S, K, 0.2, 1.0, 1.0, X, seed, persistent=persistent, log_every=log_every)
    g.run(n)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, n)
    got = g.snapshot()
    assert np.array_equal(got, o), f"{int((got != o).sum())} sites differ"
    g.run(2).run(1)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 3, mcs_begin=n)
    assert np.array_equal(g.snapshot(), o)
    c, mcs = g.counts()
    assert mcs == n + 3 and np.array_equal(c, O.counts(o, S))


@pytest.mark.parametrize("L,S,ctas,log_every", [(128, 3, 8, 3), (256, 5, 6, 2), (384, 3, 8, 10), (1024, 3, 5, 10)])
def test_flag_kernel_128_thread_ctas(L, S, ctas, log_every):
    """The flag kernel with more than 4 CTAs per SM on a uniform one-byte
    lattice runs its 128-thread build (two quads per thread, stepped
    pairwise): bit-exact after every MCS, fused counts included."""
    K = (1,) if S == 3 else (1, 2)
    X = 2.0 + L / 64
    seed = 515 + L
    g, o, D = _pair(L, S, K, 0.2, 1.0, 1.0, X, seed, persistent=3, ctas_per_sm=ctas, log_every=log_every)
    assert g.update_kernel == "persistent_kernel"
    for m in range(4):
        g.run(1)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=m)
        assert np.array_equal(g.snapshot(), o), m
    g.run(11)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 11, mcs_begin=4)
    assert np.array_equal(g.snapshot(), o)
    ms, log = g.counts_log()
    _, olog, _ = O.run_observed(O.init(L, S, 0.2, seed), D, 1.0, 1.0, X, seed, 15, log_every=log_every)
    assert np.array_equal(log, olog)


def test_flag_kernel_128_thread_default_on_deep_phases():
    """L = 6400 (2500 blocks per coarse phase): persistent = 1 runs the flag
    kernel's 128-thread build; bit-exact against the oracle after 2 MCS."""
    L, S, seed = 6400, 3, 6400
    X = 2.0 * 1e-4 * L * L
    g, o, D = _pair(L, S, (1,), 0.25, 1.0, 1.0, X, seed)
    assert g.update_kernel == "persistent_kernel"
    g.run(2)
    o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 2)
    assert np.array_equal(g.snapshot(), o)


def test_cfg1_competition_only_L64():
    w = W.CFG1
    g, o, D = _pair(w.L, w.S, w.K, w.p_empty, w.interact, w.reproduce, w.exchange, w.seed)
    for m in range(w.n_mcs):
        g.run(1)
        o, _ = O.replay_run(o, D, w.interact, w.reproduce, w.exchange, w.seed, 1, mcs_begin=m)
        assert np.array_equal(g.snapshot(), o), m


def test_cfg2_rpsls_L800_every_mcs():
    w = W.CFG2
    X = _x(w.L, w.mobility, w.exchange)
    assert X == E.exchange_from_mobility(w.mobility, w.L * w.L) == pytest.approx(128.0)
    g, o, D = _pair(w.L, w.S, w.K, w.p_empty, w.interact, w.reproduce, X, w.seed)
    for m in range(w.n_mcs):
        g.run(1)
        o, _ = O.replay_run(o, D, w.interact, w.reproduce, X, w.seed, 1, mcs_begin=m)
        if m < 20 or m % 25 == 24 or m == w.n_mcs - 1:
            assert np.array_equal(g.snapshot(), o), m
    assert np.array_equal(g.snapshot(), o)


@pytest.mark.parametrize("M", [1e-5, 1e-4, 1e-3])
def test_cfg3_L3200_full_size(M):
    """Full-size lattice in the benchmark's launch configuration (persistent
    kernel, chunks ending at log points every 10 MCS), checked at MCS 1, 2,
    10 and 100 (M = 1e-4; about 35 s of replay oracle) and 1, 3, 10 (the two
    other mobilities)."""
    w = W.CFG3[M]
    X = _x(w.L, w.mobility, w.exchange)
    g, o, D = _pair(w.L, w.S, w.K, w.p_empty, w.interact, w.reproduce, X, w.seed,
                    log_every=w.log_every)
    checkpoints = [1, 2, 10, 100] if M == 1e-4 else [1, 3, 10]
    m = 0
    for c in checkpoints:
        g.run(c - m)
        o, _ = O.replay_run(o, D, w.interact, w.reproduce, X, w.seed, c - m, mcs_begin=m)
        m = c
        assert np.array_equal(g.snapshot(), o), (M, c)
    ms, log = g.counts_log()
    assert list(ms) == list(range(0, m + 1, 10))
    assert np.array_equal(log[-1], O.counts(o, w.S))


def test_counts_log_matches_oracle():
    L, S, K, I, P, X, seed = 40, 5, (1, 2), 1.0, 1.0, 3.0, 77
    g, o, D = _pair(L, S, K, 0.2, I, P, X, seed, log_every=4)
    g.run(10).run(9)
    lat, log, mend = O.run_observed(o, D, I, P, X, seed, 19, log_every=4)
    ms, glog = g.counts_log()
    assert list(ms) == [0, 4, 8, 12, 16] and mend == 19
    assert np.array_equal(glog, log)
    assert np.array_equal(g.snapshot(), lat)


@pytest.mark.parametrize("L,S,log_every", [(128, 3, 1), (128, 5, 7), (192, 3, 3), (256, 5, 2),
                                           (67, 3, 5)])
def test_fused_counts_log_matches_oracle(L, S, log_every):
    """Counts of log points fused into the persistent kernel (each site
    counted by the last block that touches it in the MCS) equal the
    oracle's histogram after that MCS; uniform (L=128, 256) and non-uniform
    partitions, several log points open in one launch."""
    K, I, P, X, seed = ((1,) if S == 3 else (1, 2)), 1.0, 1.0, 2.0 + L / 64, 4242 + L
    g, o, D = _pair(L, S, K, 0.2, I, P, X, seed, log_every=log_every)
    n = 6 * log_every + 1
    g.run(n)
    lat, log, mend = O.run_observed(o, D, I, P, X, seed, n, log_every=log_every)
    ms, glog = g.counts_log()
    assert list(ms) == list(range(0, n + 1, log_every))
    assert np.array_equal(glog, log)
    assert np.array_equal(g.snapshot(), lat)
    assert g.mcs == n


@pytest.mark.parametrize("L,persistent", [(16, True), (16, False), (128, True), (128, 5), (128, 6)])
def test_stop_at_extinction_matches_oracle(L, persistent):
    S, K, I, P = 3, (1,), 1.0, 1.0
    seed = 5 if L == 16 else 6   # both go extinct within the budget
    X = O.exchange_from_mobility(0.1 if L == 16 else 3e-4, L * L)
    g, o, D = _pair(L, S, K, 0.25, I, P, X, seed, log_every=10, stop_at_extinction=True,
                    persistent=persistent)
    g.run(3000)
    lat, log, mend = O.run_observed(o, D, I, P, X, seed, 3000, log_every=10, stop_at_extinction=True)
    assert mend < 3000
    assert g.mcs == mend
    assert np.array_equal(g.snapshot(), lat)
    ms, glog = g.counts_log()
    assert np.array_equal(glog, log) and ms[-1] == mend


def test_restore_resume_exact():
    L, S, K, I, P, X, seed = 100, 3, (1,), 1.0, 1.0, 2.0, 9
    g, o, D = _pair(L, S, K, 0.25, I, P, X, seed, log_every=10)
    g.run(7)
    snap7 = g.snapshot()
    g.run(6)
    full = g.snapshot()
    h = E.Lattice(L, S, E.circulant(S, K), (I, P, X), seed, p_empty=0.25, log_every=10)
    h.restore(snap7, 7)
    assert h.mcs == 7
    h.run(6)
    assert np.array_equal(h.snapshot(), full)
    ref, _ = O.replay_run(snap7, D, I, P, X, seed, 6, mcs_begin=7)
    assert np.array_equal(full, ref)


@pytest.mark.parametrize("L,persistent", [(128, 1), (256, 1), (128, 3), (128, 5), (384, 5), (128, 6), (256, 6)])
def test_restore_other_lattice_at_same_mcs(L, persistent):
    """A different lattice restored at an MCS the handle has already run
    through: nothing left on the device by the earlier run (boundary records,
    epochs) may reach the new one."""
    S, D, seed = 3, E.circulant(3, [1]), 41
    g = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25, persistent=persistent)
    for n in (1, 2, 3):
        for k in range(2):
            lat = O.init(L, S, 0.25, 1000 + 10 * n + k)
            g.restore(lat, 0)
            g.run(n)
            ref, _ = O.replay_run(lat, O.circulant(S, [1]), 1.0, 1.0, 2.0, seed, n)
            assert np.array_equal(g.snapshot(), ref), (n, k)


def test_step_host_end_to_end():
    L, S, K, I, P, X, seed = 64, 5, (1, 2), 1.0, 1.0, 1.5, 21
    g, o, D = _pair(L, S, K, 0.2, I, P, X, seed)
    out, counts = g.step_host(o, 0, 5)
    ref, _ = O.replay_run(o, D, I, P, X, seed, 5)
    assert np.array_equal(out, ref)
    assert np.array_equal(counts, O.counts(ref, S))
    out2, _ = g.step_host(out, 5, 3)
    ref2, _ = O.replay_run(ref, D, I, P, X, seed, 3, mcs_begin=5)
    assert np.array_equal(out2, ref2)


def test_torch_buffer_and_stream_interop():
    import torch
    L, S, K, I, P, X, seed = 96, 3, (1,), 1.0, 1.0, 1.0, 33
    buf = torch.zeros(E.lattice_bytes(L), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    g = E.Lattice(L, S, E.circulant(S, K), (I, P, X), seed, p_empty=0.25, stream=stream,
                  device_buffer=buf)
    g.run(4)
    g.sync()
    view = g.as_tensor()[:, :L].cpu().numpy()
    o, _ = O.replay_run(O.init(L, S, 0.25, seed), O.circulant(S, K), I, P, X, seed, 4)
    assert np.array_equal(view, o)
    assert np.array_equal(g.snapshot(), o)
    assert g.stream_ptr == stream.cuda_stream


def test_launch_modes_agree_and_chunking_is_invisible():
    L, S, K, I, P, X, seed = 150, 5, (1, 2), 1.0, 1.0, 5.0, 55
    a = E.Lattice(L, S, E.circulant(S, K), (I, P, X), seed, p_empty=0.2, persistent=True, log_every=7)
    b = E.Lattice(L, S, E.circulant(S, K), (I, P, X), seed, p_empty=0.2, persistent=False, log_every=5)
    a.run(3).run(11).run(1)
    b.run(15)
    assert np.array_equal(a.snapshot(), b.snapshot())
    assert a.launches > 0 and b.launches > a.launches


@pytest.mark.parametrize("persistent", [3, 6], ids=["flags", "mailbox"])
def test_bounded_wait_times_out_with_status(persistent):
    """A block whose epoch or records are never published (host-controlled
    hook: the flag nothing sets) makes its neighbours' bounded waits run out;
    the kernel returns, escg_sync reports ESCG_ETIMEOUT and the handle
    refuses to run until a lattice is restored.  No hang, no fault."""
    L, S = 256, 3
    g = E.Lattice(L, S, E.circulant(S, [1]), (1.0, 1.0, 1.0), 3, p_empty=0.25, persistent=persistent)
    ref = g.snapshot()
    g.debug_stall_block(0, spin_limit=2000)
    g.run(3)
    with pytest.raises(E.EscgError) as ei:
        g.sync()
    assert ei.value.status == -5
    with pytest.raises(E.EscgError) as ei2:
        g.run(1)
    assert ei2.value.status == -4
    g.debug_stall_block(-1)
    g.restore(ref, 0)
    g.run(2)
    o, _ = O.replay_run(ref, O.circulant(S, [1]), 1.0, 1.0, 1.0, 3, 2)
    assert np.array_equal(g.snapshot(), o)


def test_kernel_timing_counts_launches():
    g = E.Lattice(64, 3, E.circulant(3, [1]), (1.0, 1.0, 1.0), 3, time_kernels=True)
    g.run(25)
    ms, n = g.kernel_time()
    assert n == 1 and ms > 0     # one persistent launch (counts fused, no stop)
    h = E.Lattice(64, 3, E.circulant(3, [1]), (1.0, 1.0, 1.0), 3, time_kernels=True,
                  stop_at_extinction=True)
    h.run(25)
    assert h.kernel_time()[1] == 3   # stasis is decided at each log point
    assert E.int_throughput()[0] > 1e12


def test_roofline_probes():
    """The denominators of the bench's rooflines: the step's instruction mix
    runs at a positive rate of at most the 128-per-SM-per-clock issue ceiling,
    and an L2-resident copy moves more than a few TB/s."""
    alg, per_sm_clk = E.alg_throughput()
    assert alg > 1e12 and 0 < per_sm_clk <= 128.5
    assert E.l2_copy_gbs(8 << 20, 20) > 1000.0


def test_restore_rejects_values_outside_states():
    L, S = 40, 3
    g = E.Lattice(L, S, E.circulant(S, [1]), (1.0, 1.0, 1.0), 3, p_empty=0.25)
    good = g.snapshot()
    bad = good.copy()
    bad[L - 1, L - 1] = S + 1
    with pytest.raises(E.EscgError) as ei:
        g.restore(bad, 0)
    assert ei.value.status == -1
    with pytest.raises(E.EscgError):
        g.run(1)
    g.restore(good, 0)
    g.run(2)
    o, _ = O.replay_run(good, O.circulant(S, [1]), 1.0, 1.0, 1.0, 3, 2)
    assert np.array_equal(g.snapshot(), o)


def test_async_host_steps_on_two_handles():
    """escg_step_host_async on two handles used alternately gives what
    escg_step_host gives; one step in flight per handle; errors surface at
    the wait."""
    torch = pytest.importorskip("torch")
    L, S, seed = 128, 3, 31
    D = E.circulant(S, [1])
    a = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25)
    b = E.Lattice(L, S, D, (1.0, 1.0, 2.0), seed, p_empty=0.25, stream=torch.cuda.Stream())
    lat = torch.from_numpy(O.init(L, S, 0.25, 77)).pin_memory().numpy()
    ref, cref = a.step_host(lat, 10, 10)
    outs = [torch.empty((L, L), dtype=torch.uint8).pin_memory().numpy() for _ in range(2)]
    cnts = [torch.zeros(S + 1, dtype=torch.int64).pin_memory().numpy().view(np.uint64) for _ in range(2)]
    hs = (a, b)
    for k in range(6):
        i = k & 1
        if k >= 2:
            hs[i].step_host_wait()
            assert np.array_equal(outs[i], ref) and np.array_equal(cnts[i], cref)
        hs[i].step_host_async(lat, 10, 10, outs[i], cnts[i])
        if k == 0:
            with pytest.raises(E.EscgError):
                a.step_host_async(lat, 10, 10, outs[0], cnts[0])   # one in flight
    for h in hs:
        h.step_host_wait()
    assert all(np.array_equal(o, ref) for o in outs)
    o, _ = O.replay_run(O.init(L, S, 0.25, 77), O.circulant(S, [1]), 1.0, 1.0, 2.0, seed, 10, mcs_begin=10)
    assert np.array_equal(ref, o)
    bad = lat.copy()
    bad[3, 4] = S + 2
    a.step_host_async(bad, 0, 5, outs[0], cnts[0])
    with pytest.raises(E.EscgError):
        a.step_host_wait()


@pytest.mark.parametrize("bits", [8, 2])
def test_maximum_size_lattice(bits):
    """The largest lattice the boundary takes (L = 16384, 268 M sites; both
    run the flag kernel's 128-thread build): bit-exact against the replay
    oracle after one MCS, and the counts add up to N."""
    L, S, seed = 16384, 3, 16384 + bits
    D = O.circulant(S, (1,))
    X = 2.0 * 1e-4 * L * L
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, bits_per_site=bits)
    o = O.init(L, S, 0.25, seed)
    assert np.array_equal(g.snapshot(), o)
    g.run(1)
    o, att = O.replay_run(o, D, 1.0, 1.0, X, seed, 1)
    assert att == L * L
    assert np.array_equal(g.snapshot(), o)
    c, m = g.counts()
    assert m == 1 and int(c.sum()) == L * L and np.array_equal(c, O.counts(o, S))
    g.close()


@pytest.mark.parametrize("persistent", [3, 0, 5], ids=["flags", "phase", "owners"])
@pytest.mark.parametrize("L,H,reflect", [(131, 131, False), (100, 100, False), (300, 140, False),
                                         (131, 137, True)])
def test_generic_staging_leaves_row_padding(L, H, reflect, persistent):
    """Generic partitions whose rows end mid-way through an 8-byte group
    (the flag and phase kernels' aligned tile staging reads whole groups;
    the block owners write back single sites at the row ends): the lattice
    stays bit-exact against the oracle after every MCS and the row padding
    beyond column L of the caller's device buffer is never written."""
    torch = pytest.importorskip("torch")
    S, seed, X = 3, 4100 + L + H, 2.5
    D = O.circulant(S, (1,))
    pitch = E.lattice_pitch(L)
    buf = torch.zeros(E.lattice_bytes(L, H), dtype=torch.uint8, device="cuda")
    g = E.Lattice(L, S, D, (1.0, 1.0, X), seed, p_empty=0.25, persistent=persistent, H=H,
                  reflecting_boundary=reflect, device_buffer=buf)
    g.sync()
    view = buf.view(H, pitch)
    view[:, L:] = 0xAB
    torch.cuda.synchronize()
    o = O.init(L, S, 0.25, seed, H=H)
    for m in range(4):
        g.run(1)
        o, _ = O.replay_run(o, D, 1.0, 1.0, X, seed, 1, mcs_begin=m, reflect=reflect)
        assert np.array_equal(g.snapshot(), o), m
    g.sync()
    pad = view[:, L:].cpu().numpy()
    assert (pad == 0xAB).all(), int((pad != 0xAB).sum())
    g.close()
