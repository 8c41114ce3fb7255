"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; host-side argument validation and helpers work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2508_16639_gb300 as E
from paper_2508_16639_gb300 import _lib
from paper_2508_16639_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(escg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 20
    handle = C.CDLL(_lib.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(handle, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert names <= set(_lib.SIGNATURES), sorted(names - set(_lib.SIGNATURES))


def test_helpers_match_oracle(lib):
    for S, K in [(3, [1]), (5, [1, 2]), (7, [1, 3]), (4, [])]:
        assert np.array_equal(E.circulant(S, K), O.circulant(S, K))
    for M, N in [(1e-4, 640000), (1e-5, 10240000), (3e-6, 123)]:
        assert E.exchange_from_mobility(M, N) == O.exchange_from_mobility(M, N)
    assert E.lattice_pitch(3200) == 3200 and E.lattice_pitch(100) == 112
    assert E.lattice_bytes(100) == 100 * 112


def _create(lib, L, S, D, rates, seed=1):
    r = _lib.Rates(*rates)
    Dc = np.ascontiguousarray(D, dtype=np.uint8)
    return lib.escg_create(L, S, Dc.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(r), seed)


@pytest.mark.parametrize("L,S,D,rates,msg", [
    (7, 3, O.circulant(3, [1]), (1, 1, 1), "L=7"),
    (16385, 3, O.circulant(3, [1]), (1, 1, 1), "L=16385"),
    (64, 1, np.zeros((1, 1)), (1, 1, 1), "S=1"),
    (64, 16, np.zeros((16, 16)), (1, 1, 1), "S=16"),
    (64, 3, np.eye(3), (1, 1, 1), "diagonal"),
    (64, 3, 2 * O.circulant(3, [1]), (1, 1, 1), "not 0 or 1"),
    (64, 3, O.circulant(3, [1]), (0, 0, 0), "rates"),
    (64, 3, O.circulant(3, [1]), (-1, 1, 1), "rates"),
    (64, 3, O.circulant(3, [1]), (float("nan"), 1, 1), "rates"),
])
def test_create_rejects_bad_arguments(lib, L, S, D, rates, msg):
    h = _create(lib, L, S, D, rates)
    assert not h
    assert msg in lib.escg_last_error().decode()


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.escg_run(None, 1) == _lib.ESCG_EINVAL
    assert lib.escg_sync(None) == _lib.ESCG_EINVAL
    out = np.zeros(4, dtype=np.uint64)
    assert lib.escg_counts(None, out.ctypes.data_as(C.POINTER(C.c_uint64)), None) == _lib.ESCG_EINVAL
    lib.escg_destroy(None)


def test_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(E.EscgError, match="no CUDA device"):
        E.Lattice(64, 3, O.circulant(3, [1]), (1, 0, 0), 1)


@pytest.mark.parametrize("bad,msg", [
    (dict(L=7), "bad L"), (dict(S=1), "bad L"), (dict(rates=(0, 0, 0)), "bad rates"),
    (dict(p_empty=1.5), "bad rates"), (dict(max_mcs=2**33), "bad rates"),
])
def test_batch_create_rejects_bad_specs(lib, bad, msg):
    spec = dict(L=64, S=3, digraph=O.circulant(3, [1]), rates=(1, 1, 1), seed=1, p_empty=0.25,
                max_mcs=100, stop_at_extinction=True)
    spec.update(bad)
    with pytest.raises(E.EscgError, match=msg):
        E.Batch([spec, dict(spec, L=64, S=3, rates=(1, 1, 1), p_empty=0.0, max_mcs=10)])


def test_packed_and_rectangular_size_helpers(lib):
    """Row pitch of a lattice stored with b bits per site: ceil(L b / 8)
    rounded up to 16 bytes; H rows of it."""
    for L in (64, 100, 131, 3200, 12800):
        for b in (8, 4, 2):
            row = -(-L * b // 8)
            assert E.lattice_pitch(L, b) == -(-row // 16) * 16
            for H in (64, 97, L):
                assert E.lattice_bytes(L, H, b) == H * E.lattice_pitch(L, b)
    assert lib.escg_lattice_pitch_ex(64, 3) == 0 and lib.escg_lattice_pitch_ex(0, 8) == 0
    assert lib.escg_lattice_pitch_ex(100, 0) == lib.escg_lattice_pitch(100)
    assert lib.escg_lattice_bytes_rect(100, 50) == 50 * 112


def _create_ex(lib, L, S, **fields):
    D = np.ascontiguousarray(O.circulant(S, [1] if S == 3 else [1, 2]), dtype=np.uint8)
    r = _lib.Rates(1.0, 1.0, 1.0)
    opt = _lib.Options()
    lib.escg_default_options(C.byref(opt))
    for k, v in fields.items():
        setattr(opt, k, v)
    return lib.escg_create_ex(L, S, D.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(r), 1, C.byref(opt))


@pytest.mark.parametrize("L,S,fields,msg", [
    (64, 3, dict(height=7), "height=7"),
    (64, 3, dict(height=16385), "height=16385"),
    (64, 3, dict(bits_per_site=3), "bits_per_site"),
    (64, 5, dict(bits_per_site=2), "S=5"),
    (48, 3, dict(bits_per_site=4), ">= 64"),
    (128, 3, dict(bits_per_site=2, height=40), ">= 64"),
    (64, 3, dict(persistent=7), "persistent"),
    (64, 3, dict(neighbourhood=6), "neighbourhood"),
    (64, 3, dict(reflecting_boundary=2), "neighbourhood"),
    (64, 3, dict(device_lattice=0x1001), "aligned"),
    (64, 3, dict(p_empty=1.5), "p_empty"),
    (64, 3, dict(autotune=2), "autotune"),
])
def test_create_rejects_bad_options(lib, L, S, fields, msg):
    """Options are checked on the host before any device work, so an invalid
    one (including a device buffer that is not 16-byte aligned) never
    reaches a kernel."""
    assert not _create_ex(lib, L, S, **fields)
    assert msg in lib.escg_last_error().decode()


@pytest.mark.parametrize("ptr,counts,L,mcs_begin,n_mcs,msg", [
    (0x1001, None, 64, 0, 1, "16-byte aligned"),
    (0x1000, 0x2004, 64, 0, 1, "8-byte aligned"),
    (0x1000, None, 4097, 0, 1, "4096"),
    (0x1000, None, 64, 1, 2**64 - 1, "2^31"),
    (0x1000, None, 64, 2**31, 0, "2^31"),
    (0x1000, None, 64, 2**31 - 5, 5, "2^31"),
])
def test_noalloc_rejects_bad_arguments_before_any_device_work(lib, ptr, counts, L, mcs_begin, n_mcs, msg):
    """escg_run_noalloc checks its arguments on the host first, so a
    misaligned buffer or an MCS range that would pass 2^31 (or wrap around
    2^64) never reaches a kernel (none of these touch the pointers)."""
    D = np.ascontiguousarray(O.circulant(3, [1]), dtype=np.uint8)
    r = _lib.Rates(1.0, 1.0, 1.0)
    rc = lib.escg_run_noalloc(C.c_void_p(ptr), L, 3, D.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(r), 1,
                              mcs_begin, n_mcs, C.c_void_p(counts) if counts else None, None)
    assert rc == _lib.ESCG_EINVAL
    assert msg in lib.escg_last_error().decode()
