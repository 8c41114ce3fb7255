"""escg_run_noalloc -- the entry point for callers that cannot let the
library allocate device memory (a fixed, pre-reserved GPU memory budget, or
loops where cudaMalloc would synchronise the device) -- produces the same
lattice and counts as the allocating path (escg_create + escg_run).

The caller (this test) owns every buffer: the lattice is a torch uint8
tensor and the counts a torch uint64 tensor.  Two calls in a row continue
the same run, so the second call also checks that the shared scratch array
is cleared between calls.  Kept in a file of its own that pytest collects
last."""
import ctypes as C

import numpy as np
import pytest

import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300 import _lib
from paper_2508_16639_gb300.build import build

pytestmark = pytest.mark.gpu


def _noalloc(lib, buf, L, S, D, rates, seed, mcs_begin, n_mcs, counts, stream):
    Dc = np.ascontiguousarray(D, dtype=np.uint8)
    r = _lib.Rates(*rates)
    return lib.escg_run_noalloc(C.c_void_p(buf.data_ptr()), L, S, Dc.ctypes.data_as(C.POINTER(C.c_uint8)),
                                C.byref(r), seed, mcs_begin, n_mcs,
                                C.c_void_p(counts.data_ptr()) if counts is not None else None,
                                C.c_void_p(stream.cuda_stream))


def _device_lattice(lat, L):
    import torch
    buf = torch.zeros((L, E.lattice_pitch(L)), dtype=torch.uint8, device="cuda")
    buf[:, :L] = torch.from_numpy(lat).cuda()
    return buf


@pytest.mark.parametrize("L,S,K,rates,calls", [
    (128, 3, (1,), (1.0, 1.0, 3.3), (5, 7)),      # uniform 64x64 blocks
    (100, 5, (1, 2), (1.0, 1.0, 2.0), (5, 7)),    # non-uniform partition
    (4096, 3, (1,), (1.0, 1.0, 2.0 * 1e-4 * 4096 ** 2), (3, 2)),   # the documented limit: 64 x 64 blocks
])
def test_noalloc_matches_allocating_entry_point(L, S, K, rates, calls):
    import torch
    build()
    lib = _lib.load()
    seed = 0x5EED0000 + L
    D = E.circulant(S, K)
    ref = E.Lattice(L, S, D, rates, seed, p_empty=0.25)
    buf = _device_lattice(ref.snapshot(), L)
    counts = torch.zeros(S + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    m = 0
    for n in calls:    # two calls in a row, the second continuing the first
        _lib.check(_noalloc(lib, buf, L, S, D, rates, seed, m, n, counts, stream))
        ref.run(n)
        m += n
        want = ref.snapshot()
        got = buf[:, :L].cpu().numpy()
        assert np.array_equal(got, want), f"lattice differs after MCS {m}"
        c, mcs = ref.counts()
        assert mcs == m
        assert np.array_equal(counts.cpu().numpy().astype(np.uint64), c)
    ref.close()


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the kernels and looks up the scratch
    array), further calls leave the device's free memory unchanged."""
    import torch
    build()
    lib = _lib.load()
    L, S, D, rates, seed = 256, 3, E.circulant(3, (1,)), (1.0, 1.0, 13.1), 7
    ref = E.Lattice(L, S, D, rates, seed, p_empty=0.25)
    buf = _device_lattice(ref.snapshot(), L)
    ref.close()
    counts = torch.zeros(S + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    _lib.check(_noalloc(lib, buf, L, S, D, rates, seed, 0, 4, counts, stream))
    free0, _ = torch.cuda.mem_get_info()
    for k in range(3):
        _lib.check(_noalloc(lib, buf, L, S, D, rates, seed, 4 + 3 * k, 3, counts, stream))
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"


def test_noalloc_rejects_a_lattice_value_outside_the_states():
    """A byte above S is refused on the device before any step (the
    transition table is indexed by the pair): ESCG_EINVAL, lattice unchanged."""
    import torch
    build()
    lib = _lib.load()
    L, S, D, rates, seed = 100, 5, E.circulant(5, (1, 2)), (1.0, 1.0, 2.0), 11
    ref = E.Lattice(L, S, D, rates, seed, p_empty=0.2)
    lat = ref.snapshot()
    ref.close()
    lat[37, 51] = S + 1
    buf = _device_lattice(lat, L)
    counts = torch.zeros(S + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    rc = _noalloc(lib, buf, L, S, D, rates, seed, 0, 3, counts, stream)
    assert rc == _lib.ESCG_EINVAL
    assert "outside 0..S" in lib.escg_last_error().decode()
    assert np.array_equal(buf[:, :L].cpu().numpy(), lat)
    # the next valid call runs normally
    lat[37, 51] = 0
    buf[:, :L] = torch.from_numpy(lat).cuda()
    torch.cuda.synchronize()
    _lib.check(_noalloc(lib, buf, L, S, D, rates, seed, 0, 3, counts, stream))


def test_noalloc_rejects_lattices_beyond_its_scratch():
    build()
    lib = _lib.load()
    D = E.circulant(3, [1])
    r = _lib.Rates(1.0, 1.0, 1.0)
    rc = lib.escg_run_noalloc(C.c_void_p(16), 4097, 3, np.ascontiguousarray(D).ctypes.data_as(
        C.POINTER(C.c_uint8)), C.byref(r), 1, 0, 1, None, None)
    assert rc == _lib.ESCG_EINVAL
    assert "4096" in lib.escg_last_error().decode()
