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
    rc = lib.escg_run_noalloc(C.c_void_p(buf.data_ptr()), L, S, Dc.ctypes.data_as(C.POINTER(C.c_uint8)),
                              C.byref(r), seed, mcs_begin, n_mcs, C.c_void_p(counts.data_ptr()),
                              C.c_void_p(stream.cuda_stream))
    _lib.check(rc)


@pytest.mark.parametrize("L,S,K,rates", [(128, 3, (1,), (1.0, 1.0, 3.3)),      # uniform 64x64 blocks
                                         (100, 5, (1, 2), (1.0, 1.0, 2.0))])  # non-uniform partition
def test_noalloc_matches_allocating_entry_point(L, S, K, rates):
    import torch
    build()
    lib = _lib.load()
    seed = 0x5EED0000 + L
    D = E.circulant(S, K)
    ref = E.Lattice(L, S, D, rates, seed, p_empty=0.25)
    lat0 = ref.snapshot()
    pitch = E.lattice_pitch(L)
    buf = torch.zeros((L, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :L] = torch.from_numpy(lat0).cuda()
    counts = torch.zeros(S + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    m = 0
    for n in (5, 7):    # two calls in a row, the second continuing the first
        _noalloc(lib, buf, L, S, D, rates, seed, m, n, counts, stream)
        ref.run(n)
        m += n
        want = ref.snapshot()
        got = buf[:, :L].cpu().numpy()
        assert np.array_equal(got, want), f"lattice differs after MCS {m}"
        c, mcs = ref.counts()
        assert mcs == m
        assert np.array_equal(counts.cpu().numpy().astype(np.uint64), c)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    build()
    lib = _lib.load()
    D = E.circulant(3, [1])
    r = _lib.Rates(1.0, 1.0, 1.0)
    rc = lib.escg_run_noalloc(C.c_void_p(1), 4097, 3, np.ascontiguousarray(D).ctypes.data_as(
        C.POINTER(C.c_uint8)), C.byref(r), 1, 0, 1, None, None)
    assert rc == _lib.ESCG_EINVAL
    assert "4096" in lib.escg_last_error().decode()
