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
