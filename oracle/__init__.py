"""CPU oracle for the ESCG Monte Carlo step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2508_16639_gb300``) never does, and the two share no
code: this package wraps ``escg_oracle.c`` (plain single-threaded C written
from the paper's Alg. 2-4 and the schedule-v1 definition) through ctypes.

Every function takes and returns numpy arrays; lattices are ``uint8`` of
shape ``(L, L)`` (row-major, value 0 = empty, 1..S = species).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "escg_oracle.c")
_HDR = os.path.join(_HERE, "escg_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

EXCHANGE, INTERACT, REPRODUCE, INTERACT_FAIL = 0, 1, 2, 3
SHUFFLE_BLOCKS, SHUFFLE_SUBS = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, strict IEEE: no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class TraceRec(C.Structure):
    _fields_ = [("mcs", C.c_uint32), ("coarse_phase", C.c_uint32), ("fine_phase", C.c_uint32),
                ("block", C.c_uint32), ("sub", C.c_uint32), ("t", C.c_uint32),
                ("site", C.c_uint32), ("nbr", C.c_uint32), ("dir", C.c_uint8),
                ("action", C.c_uint8), ("pad", C.c_uint8 * 2)]


TRACE_DTYPE = np.dtype([("mcs", "<u4"), ("coarse_phase", "<u4"), ("fine_phase", "<u4"),
                        ("block", "<u4"), ("sub", "<u4"), ("t", "<u4"), ("site", "<u4"),
                        ("nbr", "<u4"), ("dir", "u1"), ("action", "u1"), ("pad", "u1", 2)])


class Variant(C.Structure):
    """orc_variant: neighbourhood 4/8, reflecting boundary, edge probabilities,
    rows of an L x H lattice (0: square)."""
    _fields_ = [("neighbourhood", C.c_int32), ("reflect", C.c_int32), ("prob", C.POINTER(C.c_double)),
                ("height", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            u8p, u32p, u64p, i32p, i64p = (P(C.c_uint8), P(C.c_uint32), P(C.c_uint64),
                                           P(C.c_int32), P(C.c_int64))
            d = C.c_double
            dp = P(C.c_double)
            vp = P(Variant)
            sig = {
                "orc_philox_many": (None, [C.c_int64, u32p, u32p, u32p]),
                "orc_circulant": (C.c_int, [C.c_int32, i32p, C.c_int32, u8p]),
                "orc_dominates": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p]),
                "orc_rule": (None, [C.c_int32, C.c_int32, u8p, u8p, u8p]),
                "orc_exchange_from_mobility": (d, [d, C.c_int64]),
                "orc_thresholds": (C.c_int, [d, d, d, u64p, u64p]),
                "orc_counts": (C.c_int, [C.c_int64, u8p, C.c_int32, u64p]),
                "orc_rs_attempts": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, d, d, d,
                                              C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, u8p]),
                "orc_rs_run": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, d, d, d,
                                         C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, u8p]),
                "orc_v1_partition": (C.c_int, [C.c_int32, i32p, i32p, i32p, i32p, i32p]),
                "orc_v1_cycles": (C.c_int, [C.c_int32, i32p, i32p]),
                "orc_init": (C.c_int, [C.c_int32, C.c_int32, d, C.c_uint64, u8p]),
                "orc_init_rect": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, d, C.c_uint64, u8p]),
                "orc_replay_run": (C.c_int, [C.c_int32, C.c_int32, u8p, d, d, d, C.c_uint64,
                                             C.c_int32, C.c_int32, C.c_uint32, C.c_uint32, u8p,
                                             C.c_uint32, C.c_uint64, P(TraceRec), C.c_int64, i64p]),
                "orc_run_observed": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, d, d, d,
                                               C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                               C.c_int32, u8p, u64p, C.c_int64, i64p, u32p]),
                "orc_pair_prob": (d, [C.c_int32, C.c_int32, C.c_int32, u8p, dp]),
                "orc_interaction_threshold": (C.c_uint64, [C.c_uint64, C.c_uint64, d]),
                "orc_rs_attempts_p": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, dp, d, d, d,
                                                C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, u8p]),
                "orc_rs_run_p": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, dp, d, d, d,
                                           C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, u8p]),
                "orc_replay_run_p": (C.c_int, [C.c_int32, C.c_int32, u8p, dp, d, d, d, C.c_uint64,
                                               C.c_int32, C.c_int32, C.c_uint32, C.c_uint32, u8p,
                                               C.c_uint32, C.c_uint64, P(TraceRec), C.c_int64, i64p]),
                "orc_run_observed_p": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, dp, d, d, d,
                                                 C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                                 C.c_int32, u8p, u64p, C.c_int64, i64p, u32p]),
                "orc_rs_attempts_v": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, vp, d, d, d,
                                                C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, u8p]),
                "orc_rs_run_v": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, vp, d, d, d,
                                           C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, u8p]),
                "orc_replay_run_v": (C.c_int, [C.c_int32, C.c_int32, u8p, vp, d, d, d, C.c_uint64,
                                               C.c_int32, C.c_int32, C.c_uint32, C.c_uint32, u8p,
                                               C.c_uint32, C.c_uint64, P(TraceRec), C.c_int64, i64p]),
                "orc_run_observed_v": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, u8p, vp, d, d, d,
                                                 C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                                 C.c_int32, u8p, u64p, C.c_int64, i64p, u32p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


# --------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of each counter row (n x 4) under each key row (n x 2)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32).reshape(-1, 2),
                                               (ctr.shape[0], 2)))
    out = np.zeros_like(ctr)
    _load().orc_philox_many(ctr.shape[0], _ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32),
                            _ptr(out, C.c_uint32))
    return out


def circulant(S: int, K) -> np.ndarray:
    """Dominance matrix of the circulant digraph C(S, K) as an S x S uint8 array."""
    K = np.ascontiguousarray(np.asarray(list(K), dtype=np.int32))
    D = np.zeros((S, S), dtype=np.uint8)
    _check(_load().orc_circulant(S, _ptr(K, C.c_int32), len(K), _ptr(D, C.c_uint8)), "circulant")
    return D


def dominates(a: int, b: int, D: np.ndarray) -> bool:
    D = np.ascontiguousarray(D, dtype=np.uint8)
    return bool(_load().orc_dominates(a, b, D.shape[0], _ptr(D, C.c_uint8)))


def rule(action: int, a: int, b: int, D: np.ndarray):
    """Alg. 3 applied to (selected, neighbour) = (a, b) under the given action."""
    D = np.ascontiguousarray(D, dtype=np.uint8)
    x = np.array([a], dtype=np.uint8)
    y = np.array([b], dtype=np.uint8)
    _load().orc_rule(action, D.shape[0], _ptr(D, C.c_uint8), _ptr(x, C.c_uint8), _ptr(y, C.c_uint8))
    return int(x[0]), int(y[0])


def exchange_from_mobility(M: float, N: int) -> float:
    return float(_load().orc_exchange_from_mobility(M, N))


def thresholds(I: float, P: float, X: float):
    tx, txi = C.c_uint64(), C.c_uint64()
    _check(_load().orc_thresholds(I, P, X, C.byref(tx), C.byref(txi)), "thresholds")
    return int(tx.value), int(txi.value)


def counts(lattice: np.ndarray, S: int) -> np.ndarray:
    lat = np.ascontiguousarray(lattice, dtype=np.uint8)
    c = np.zeros(S + 1, dtype=np.uint64)
    _check(_load().orc_counts(lat.size, _ptr(lat, C.c_uint8), S, _ptr(c, C.c_uint64)), "counts")
    return c


def _prob(prob, S):
    """Edge probabilities as a contiguous S x S float64 array, or None."""
    if prob is None:
        return None
    a = np.ascontiguousarray(np.asarray(prob, dtype=np.float64).reshape(S, S))
    return a


def _pp(a):
    return None if a is None else _ptr(a, C.c_double)


def _variant(S, neighbourhood, reflect, prob, height=0):
    """(Variant, keep-alive array) for the _v entry points."""
    pr = _prob(prob, S)
    v = Variant(int(neighbourhood), int(bool(reflect)), _pp(pr), int(height))
    return v, pr


def pair_prob(a: int, b: int, D: np.ndarray, prob=None) -> float:
    """Probability of the interaction of the pair (selected a, neighbour b)."""
    D = np.ascontiguousarray(D, dtype=np.uint8)
    pr = _prob(prob, D.shape[0])
    return float(_load().orc_pair_prob(a, b, D.shape[0], _ptr(D, C.c_uint8), _pp(pr)))


def interaction_threshold(TX: int, TXI: int, p: float) -> int:
    return int(_load().orc_interaction_threshold(TX, TXI, p))


def rs_attempts(lattice, D, I, P, X, seed, n_attempts, stream=0, mcs=0, prob=None, neighbourhood=4,
                reflect=False):
    """n_attempts random-sequential elementary steps (Alg. 3) in place;
    prob: optional S x S edge probabilities (Park, Chen, Szolnoki);
    neighbourhood 4 or 8, reflect: reflecting instead of periodic boundary."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8)
    H, L = lat.shape
    D = np.ascontiguousarray(D, dtype=np.uint8)
    v, _keep = _variant(D.shape[0], neighbourhood, reflect, prob)
    _check(_load().orc_rs_attempts_v(L, H, D.shape[0], _ptr(D, C.c_uint8), C.byref(v), I, P, X, seed, stream,
                                     mcs, n_attempts, _ptr(lat, C.c_uint8)), "rs_attempts")
    return lat


def rs_run(lattice, D, I, P, X, seed, n_mcs, mcs_begin=0, stream=0, prob=None, neighbourhood=4, reflect=False):
    """n_mcs random-sequential MCS (Alg. 4: N elementary steps each)."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).copy()
    H, L = lat.shape
    D = np.ascontiguousarray(D, dtype=np.uint8)
    v, _keep = _variant(D.shape[0], neighbourhood, reflect, prob)
    _check(_load().orc_rs_run_v(L, H, D.shape[0], _ptr(D, C.c_uint8), C.byref(v), I, P, X, seed, stream,
                                mcs_begin, n_mcs, _ptr(lat, C.c_uint8)), "rs_run")
    return lat


def v1_partition(L: int):
    """(coarse_start[P+1], fine_start[GQ+1], fine_of_coarse[P+1]) of schedule v1."""
    lib = _load()
    P, GQ = C.c_int32(), C.c_int32()
    _check(lib.orc_v1_partition(L, C.byref(P), C.byref(GQ), None, None, None), "v1_partition")
    cs = np.zeros(P.value + 1, dtype=np.int32)
    fs = np.zeros(GQ.value + 1, dtype=np.int32)
    fc = np.zeros(P.value + 1, dtype=np.int32)
    lib.orc_v1_partition(L, None, None, _ptr(cs, C.c_int32), _ptr(fs, C.c_int32), _ptr(fc, C.c_int32))
    return cs, fs, fc


def v1_cycles(L: int):
    G, F = C.c_int32(), C.c_int32()
    _check(_load().orc_v1_cycles(L, C.byref(G), C.byref(F)), "v1_cycles")
    return G.value, F.value


def init(L: int, S: int, p_empty: float, seed: int, H: int = None) -> np.ndarray:
    """Initial lattice of H rows (default L) and L columns, shape (H, L)."""
    H = L if H is None else H
    lat = np.zeros((H, L), dtype=np.uint8)
    _check(_load().orc_init_rect(L, H, S, p_empty, seed, _ptr(lat, C.c_uint8)), "init")
    return lat


def replay_run(lattice, D, I, P, X, seed, n_mcs, mcs_begin=0, G=None, F=None, flags=0,
               shuffle_seed=0, trace_cap=0, prob=None, neighbourhood=4, reflect=False):
    """Schedule-v1 replay of an (H, L) lattice.  Returns (lattice, attempts[, trace])."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).copy()
    H, L = lat.shape
    if G is None or F is None:
        G0, F0 = v1_cycles(L)
        G = G0 if G is None else G
        F = F0 if F is None else F
    D = np.ascontiguousarray(D, dtype=np.uint8)
    att = C.c_int64()
    tr = (TraceRec * trace_cap)() if trace_cap else None
    v, _keep = _variant(D.shape[0], neighbourhood, reflect, prob, H)
    _check(_load().orc_replay_run_v(L, D.shape[0], _ptr(D, C.c_uint8), C.byref(v), I, P, X, seed, G, F,
                                    mcs_begin, n_mcs, _ptr(lat, C.c_uint8), flags, shuffle_seed,
                                    tr, trace_cap, C.byref(att)), "replay_run")
    if trace_cap:
        n = min(att.value, trace_cap)
        arr = np.frombuffer(tr, dtype=TRACE_DTYPE, count=n).copy()
        return lat, att.value, arr
    return lat, att.value


def run_observed(lattice, D, I, P, X, seed, n_mcs, log_every=1, stop_at_extinction=False,
                 mcs_begin=0, use_rs=False, prob=None, neighbourhood=4, reflect=False):
    """Run an (H, L) lattice with counts logged every log_every MCS; returns
    (lattice, log, mcs_end)."""
    lat = np.ascontiguousarray(lattice, dtype=np.uint8).copy()
    H, L = lat.shape
    S = D.shape[0]
    D = np.ascontiguousarray(D, dtype=np.uint8)
    cap = n_mcs // log_every + 2
    log = np.zeros((cap, S + 1), dtype=np.uint64)
    nl, mend = C.c_int64(), C.c_uint32()
    v, _keep = _variant(S, neighbourhood, reflect, prob, H)
    _check(_load().orc_run_observed_v(int(use_rs), L, S, _ptr(D, C.c_uint8), C.byref(v), I, P, X, seed,
                                      mcs_begin, n_mcs, log_every, int(stop_at_extinction),
                                    _ptr(lat, C.c_uint8), _ptr(log, C.c_uint64), cap,
                                    C.byref(nl), C.byref(mend)), "run_observed")
    return lat, log[:min(nl.value, cap)], mend.value
