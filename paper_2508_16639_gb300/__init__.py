"""GB300-native Monte Carlo step of the Evolutionary Spatial Cyclic Game
(arXiv 2508.16639): Python binding of libescg.

The binding only marshals arguments into the C ABI (include/escg.h); every
step of the lattice update runs in the library's CUDA kernels.  PyTorch, when
used, supplies device memory (a uint8 tensor passed as the lattice buffer)
and the CUDA stream.  There is no CPU fallback: a missing library or device
raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (BatchOptions, EscgError, Options, Rates, ReplicaSpec, ServerOptions, check,
                   load)

__all__ = ["Lattice", "Batch", "Server", "circulant", "exchange_from_mobility", "lattice_pitch", "lattice_bytes",
           "int_throughput", "EscgError", "load"]


def _u8(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def circulant(S: int, K) -> np.ndarray:
    """Dominance digraph of the circulant graph C(S, K) (S x S uint8)."""
    K = np.ascontiguousarray(np.asarray(list(K), dtype=np.int32))
    D = np.zeros((S, S), dtype=np.uint8)
    check(load().escg_circulant(S, K.ctypes.data_as(C.POINTER(C.c_int32)), len(K), _u8(D)))
    return D


def exchange_from_mobility(M: float, N: int) -> float:
    """epsilon = 2 M N."""
    return float(load().escg_exchange_from_mobility(M, N))


def int_throughput():
    """Measured integer-instruction issue rate of the current GPU:
    (instructions/s, instructions per SM per clock)."""
    a, b = C.c_double(), C.c_double()
    check(load().escg_diag_int_throughput(C.byref(a), C.byref(b)))
    return float(a.value), float(b.value)


def alg_throughput():
    """Measured throughput of the elementary step's integer-instruction mix
    (24 per step): (instructions/s, instructions per SM per clock)."""
    a, b = C.c_double(), C.c_double()
    check(load().escg_diag_alg_throughput(C.byref(a), C.byref(b)))
    return float(a.value), float(b.value)


def l2_copy_gbs(nbytes: int, reps: int = 200) -> float:
    """Device copy bandwidth (read + write GB/s) between two L2-resident
    buffers of nbytes each."""
    g = C.c_double()
    check(load().escg_diag_l2_copy(nbytes, reps, C.byref(g)))
    return float(g.value)


def lattice_pitch(L: int, bits_per_site: int = 8) -> int:
    return int(load().escg_lattice_pitch_ex(L, bits_per_site))


def lattice_bytes(L: int, H: int = None, bits_per_site: int = 8) -> int:
    """Device bytes of an L x H lattice (H rows of lattice_pitch(L, bits) bytes)."""
    return int(load().escg_lattice_bytes_ex(L, L if H is None else H, bits_per_site))


class Lattice:
    """One lattice of L columns and H rows (default H = L) resident on the
    GPU (a handle of the C ABI); host-side arrays have shape (H, L).

    rates: (interact, reproduce, exchange).  device_buffer: optional torch
    uint8 CUDA tensor of at least lattice_bytes(L) bytes used as the lattice
    storage; stream: optional torch.cuda.Stream (or raw cudaStream_t int).
    persistent: 1 persistent dataflow launches (default; the kernel is
    picked by lattice size), 3 with epoch flags only, 2 with a TMA producer
    warp, 6 with boundary records (mailbox), 4 the whole
    lattice resident in one CTA's shared memory (small lattices; larger ones
    run as 3), 5 one CTA per 2x2 group of blocks with its tiles resident
    (any partition of the von Neumann rule whose grid the device holds;
    others run as 3), 0 one launch per coarse phase -- all bit-identical.
    autotune: with persistent = 1, time the distinct launch modes and CTA
    counts on the first handle of its size and rule and keep the fastest
    (cached for the process; see autotune_result).  dominance_prob: optional S x S edge
    probabilities (Park, Chen and Szolnoki's probabilistic dominance);
    neighbourhood 4 or 8 (Moore) and reflecting_boundary: the paper's rule
    variants.  H: rows (default L).  bits_per_site: device storage, 8 (one
    byte per site), 4 or 2 (bit-packed rows; 2 needs S <= 3)."""

    def __init__(self, L: int, S: int, digraph, rates, seed: int, p_empty: float = 0.0,
                 log_every: int = 10, stop_at_extinction: bool = False, persistent: int = 1,
                 stream=None, device_buffer=None, time_kernels: bool = False, ctas_per_sm: int = 0,
                 dominance_prob=None, neighbourhood: int = 4, reflecting_boundary: bool = False,
                 H: int = None, bits_per_site: int = 8, autotune: bool = False):
        lib = load()
        self.L, self.S = int(L), int(S)
        self.H = self.L if H is None else int(H)
        D = np.ascontiguousarray(np.asarray(digraph, dtype=np.uint8).reshape(S, S))
        r = Rates(*[float(x) for x in rates])
        opt = Options()
        lib.escg_default_options(C.byref(opt))
        opt.p_empty = float(p_empty)
        opt.log_every = int(log_every)
        opt.stop_at_extinction = int(bool(stop_at_extinction))
        opt.persistent = int(persistent)
        opt.time_kernels = int(bool(time_kernels))
        opt.ctas_per_sm = int(ctas_per_sm)
        opt.neighbourhood = int(neighbourhood)
        opt.reflecting_boundary = int(bool(reflecting_boundary))
        opt.height = self.H
        opt.bits_per_site = int(bits_per_site)
        opt.autotune = int(bool(autotune))
        self.bits_per_site = int(bits_per_site)
        if dominance_prob is not None:
            Pd = np.ascontiguousarray(np.asarray(dominance_prob, dtype=np.float64).reshape(S, S))
            opt.dominance_prob = Pd.ctypes.data_as(C.POINTER(C.c_double))   # read during creation
        if stream is not None:
            opt.cuda_stream = int(getattr(stream, "cuda_stream", stream))
        self._buffer = device_buffer  # keep the torch tensor alive
        if device_buffer is not None:
            if device_buffer.numel() * device_buffer.element_size() < lattice_bytes(L, self.H, bits_per_site):
                raise ValueError("device_buffer is smaller than lattice_bytes(L, H, bits_per_site)")
            opt.device_lattice = int(device_buffer.data_ptr())
        h = lib.escg_create_ex(self.L, self.S, _u8(D), C.byref(r), C.c_uint64(seed & (2**64 - 1)),
                               C.byref(opt))
        if not h:
            raise EscgError(-1, lib.escg_last_error().decode(errors="replace"))
        self._h = C.c_void_p(h)
        self.pitch = lattice_pitch(L, bits_per_site)

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().escg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- operations -----------------------------------------------------------
    def run(self, n_mcs: int):
        check(load().escg_run(self._h, int(n_mcs)))
        return self

    def sync(self):
        check(load().escg_sync(self._h))

    def counts(self):
        out = np.zeros(self.S + 1, dtype=np.uint64)
        mcs = C.c_uint64()
        check(load().escg_counts(self._h, out.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(mcs)))
        return out, int(mcs.value)

    def counts_log(self, cap: int = 4096):
        out = np.zeros((cap, self.S + 1), dtype=np.uint64)
        ms = np.zeros(cap, dtype=np.uint64)
        n = C.c_int64()
        check(load().escg_counts_log(self._h, out.ctypes.data_as(C.POINTER(C.c_uint64)),
                                     ms.ctypes.data_as(C.POINTER(C.c_uint64)), cap, C.byref(n)))
        return ms[:n.value].astype(np.int64), out[:n.value]

    def snapshot(self) -> np.ndarray:
        out = np.empty((self.H, self.L), dtype=np.uint8)
        check(load().escg_snapshot(self._h, _u8(out)))
        return out

    def restore(self, lattice: np.ndarray, mcs: int):
        lat = np.ascontiguousarray(lattice, dtype=np.uint8)
        if lat.shape != (self.H, self.L):
            raise ValueError("lattice shape mismatch")
        check(load().escg_restore(self._h, _u8(lat), int(mcs)))

    def step_host(self, lattice_in: np.ndarray, mcs: int, n_mcs: int, out: np.ndarray | None = None):
        """End-to-end host call: lattice in, n_mcs on the GPU, lattice and
        counts out (host buffers, copies included)."""
        lat = np.ascontiguousarray(lattice_in, dtype=np.uint8)
        if lat.shape != (self.H, self.L):
            raise ValueError("lattice shape mismatch")
        out = np.empty_like(lat) if out is None else out
        if out.shape != lat.shape or out.dtype != np.uint8 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous uint8 array of the lattice's shape")
        counts = np.zeros(self.S + 1, dtype=np.uint64)
        check(load().escg_step_host(self._h, _u8(lat), int(mcs), int(n_mcs), _u8(out),
                                    counts.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out, counts

    def step_host_async(self, lattice_in: np.ndarray, mcs: int, n_mcs: int, out: np.ndarray,
                        counts: np.ndarray):
        """step_host without waiting: the arrays (C-contiguous; pinned, e.g.
        from torch's pin_memory, for the copies to overlap other work) must
        stay alive and unread until step_host_wait()."""
        for arr, dt in ((lattice_in, np.uint8), (out, np.uint8), (counts, np.uint64)):
            if arr.dtype != dt or not arr.flags.c_contiguous:
                raise ValueError("arrays must be C-contiguous uint8 lattices and uint64 counts")
        if lattice_in.shape != (self.H, self.L) or out.shape != (self.H, self.L) or counts.size < self.S + 1:
            raise ValueError("array shapes do not match the lattice")
        self._inflight = (lattice_in, out, counts)   # keep the buffers alive
        check(load().escg_step_host_async(self._h, _u8(lattice_in), int(mcs), int(n_mcs), _u8(out),
                                          counts.ctypes.data_as(C.POINTER(C.c_uint64))))

    def step_host_wait(self):
        check(load().escg_step_host_wait(self._h))
        self._inflight = None

    def kernel_time(self, reset: bool = False):
        """(total ms, launches) of the lattice-update kernels, measured with
        CUDA events on the handle's stream (needs time_kernels=True)."""
        ms, n = C.c_double(), C.c_uint64()
        check(load().escg_kernel_time(self._h, C.byref(ms), C.byref(n), int(bool(reset))))
        return float(ms.value), int(n.value)

    @property
    def autotune_result(self):
        """(launch mode, CTAs per SM, ms per MCS, configurations timed) of a
        handle created with autotune=True; 0 configurations timed means the
        choice came from the process's cache."""
        mode, ctas, n = C.c_int32(), C.c_int32(), C.c_int32()
        ms = C.c_double()
        check(load().escg_autotune_result(self._h, C.byref(mode), C.byref(ctas), C.byref(ms), C.byref(n)))
        return int(mode.value), int(ctas.value), float(ms.value), int(n.value)

    def debug_stall_block(self, block: int, spin_limit: int = 0):
        """Test hook: never publish the epoch of one coarse block so that the
        persistent kernel's bounded waits run out (block < 0 clears it)."""
        check(load().escg_debug_stall_block(self._h, int(block), int(spin_limit)))

    @property
    def coarse_blocks(self) -> int:
        return int(load().escg_coarse_blocks(self._h))

    @property
    def update_kernel(self) -> str:
        """Name of the kernel that advances this lattice (fixed at creation)."""
        return load().escg_update_kernel(self._h).decode()

    @property
    def mcs(self) -> int:
        return int(load().escg_current_mcs(self._h))

    @property
    def launches(self) -> int:
        return int(load().escg_launch_count(self._h))

    @property
    def device_ptr(self) -> int:
        return int(load().escg_device_lattice(self._h))

    @property
    def stream_ptr(self) -> int:
        return int(load().escg_stream(self._h) or 0)

    def as_tensor(self):
        """torch view of the device lattice (H x pitch uint8), when the
        lattice lives in a torch-allocated buffer."""
        if self._buffer is None:
            raise RuntimeError("lattice storage is library-owned; pass device_buffer= to get a view")
        return self._buffer.view(-1)[: self.H * self.pitch].view(self.H, self.pitch)


def _replica_spec(sp, keep):
    """Fills a ReplicaSpec from a dict; `keep` holds the digraph array alive."""
    r = ReplicaSpec()
    D = np.ascontiguousarray(np.asarray(sp["digraph"], dtype=np.uint8))
    keep.append(D)
    r.L, r.S = int(sp["L"]), int(sp["S"])
    r.digraph = _u8(D)
    r.rates = Rates(*[float(x) for x in sp["rates"]])
    r.seed = int(sp["seed"]) & (2**64 - 1)
    r.p_empty = float(sp.get("p_empty", 0.0))
    r.max_mcs = int(sp["max_mcs"])
    r.stop_at_extinction = int(bool(sp.get("stop_at_extinction", False)))
    if sp.get("dominance_prob") is not None:
        Pd = np.ascontiguousarray(np.asarray(sp["dominance_prob"], dtype=np.float64).reshape(r.S, r.S))
        keep.append(Pd)
        r.dominance_prob = Pd.ctypes.data_as(C.POINTER(C.c_double))
    return r


class Batch:
    """An ensemble of independent replicas run together on the GPU (a batch
    handle of the C ABI).  specs: sequence of dicts with keys L, S, digraph,
    rates (interact, reproduce, exchange), seed, p_empty, max_mcs,
    stop_at_extinction.  threads: CTA size (64/128/256) or 0 to autotune.
    resident: replicas that fit one CTA's shared memory keep their whole
    lattice there for each chunk (default False: the block-by-block chunk
    kernel, faster for every size measured)."""

    def __init__(self, specs, log_every: int = 10, threads: int = 0, use_graph: bool = True,
                 stream=None, resident: bool = False):
        lib = load()
        self.n = len(specs)
        self._digraphs = []
        arr = (ReplicaSpec * self.n)()
        self.L, self.S = [], []
        keep = self._digraphs
        for i, sp in enumerate(specs):
            arr[i] = _replica_spec(sp, keep)
            self.L.append(int(sp["L"]))
            self.S.append(int(sp["S"]))
        opt = BatchOptions()
        lib.escg_batch_default_options(C.byref(opt))
        opt.log_every = int(log_every)
        opt.threads = int(threads)
        opt.use_graph = int(bool(use_graph))
        opt.resident = int(bool(resident))
        if stream is not None:
            opt.cuda_stream = int(getattr(stream, "cuda_stream", stream))
        h = lib.escg_batch_create(self.n, arr, C.byref(opt))
        if not h:
            raise EscgError(-1, lib.escg_last_error().decode(errors="replace"))
        self._h = C.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            load().escg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, max_mcs: int = 0):
        check(load().escg_batch_run(self._h, int(max_mcs)))
        return self

    def sync(self):
        check(load().escg_batch_sync(self._h))

    def status(self):
        """(mcs[n], extinct[n], counts[n, 16]) -- counts at each replica's
        last log point."""
        mcs = np.zeros(self.n, dtype=np.uint64)
        ext = np.zeros(self.n, dtype=np.int32)
        cnt = np.zeros((self.n, 16), dtype=np.uint64)
        check(load().escg_batch_status(self._h, mcs.ctypes.data_as(C.POINTER(C.c_uint64)),
                                       ext.ctypes.data_as(C.POINTER(C.c_int32)),
                                       cnt.ctypes.data_as(C.POINTER(C.c_uint64))))
        return mcs.astype(np.int64), ext.astype(bool), cnt

    def snapshot(self, i: int) -> np.ndarray:
        out = np.empty((self.L[i], self.L[i]), dtype=np.uint8)
        check(load().escg_batch_snapshot(self._h, int(i), _u8(out)))
        return out

    @property
    def active(self) -> int:
        return int(load().escg_batch_active(self._h))

    @property
    def threads(self) -> int:
        return int(load().escg_batch_threads(self._h))

    @property
    def uses_tma(self) -> bool:
        return bool(load().escg_batch_uses_tma(self._h))

    @property
    def launches(self) -> int:
        return int(load().escg_batch_launch_count(self._h))


class Server:
    """Continuous-batching request loop (a server handle of the C ABI).
    submit() queues a run (same dict as Batch specs) and returns its id;
    step() admits queued runs while slots and device memory allow, advances
    every resident run by chunks_per_step * log_every MCS, and retires the
    finished ones; poll() lists runs finished since the last poll."""

    def __init__(self, arena_bytes: int = 256 << 20, max_slots: int = 1024, log_every: int = 10,
                 threads: int = 0, chunks_per_step: int = 4, keep_lattice: bool = False, stream=None):
        lib = load()
        opt = ServerOptions()
        lib.escg_server_default_options(C.byref(opt))
        opt.arena_bytes = int(arena_bytes)
        opt.max_slots = int(max_slots)
        opt.log_every = int(log_every)
        opt.threads = int(threads)
        opt.chunks_per_step = int(chunks_per_step)
        opt.keep_lattice = int(bool(keep_lattice))
        if stream is not None:
            opt.cuda_stream = int(getattr(stream, "cuda_stream", stream))
        h = lib.escg_server_create(C.byref(opt))
        if not h:
            raise EscgError(-1, lib.escg_last_error().decode(errors="replace"))
        self._h = C.c_void_p(h)
        self._L = {}

    def close(self):
        if getattr(self, "_h", None):
            load().escg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, spec) -> int:
        keep = []
        r = _replica_spec(spec, keep)
        rid = int(load().escg_server_submit(self._h, C.byref(r)))
        if rid < 0:
            check(rid)
        self._L[rid] = int(spec["L"])
        return rid

    def step(self) -> int:
        n = C.c_int32()
        check(load().escg_server_step(self._h, C.byref(n)))
        return int(n.value)

    def cancel(self, rid: int):
        """Cancel a queued or running run between steps (see escg_server_cancel)."""
        check(load().escg_server_cancel(self._h, int(rid)))

    def poll(self, cap: int = 65536):
        ids = np.zeros(cap, dtype=np.int64)
        n = C.c_int32()
        check(load().escg_server_poll(self._h, ids.ctypes.data_as(C.POINTER(C.c_int64)), cap, C.byref(n)))
        return [int(x) for x in ids[:n.value]]

    def result(self, rid: int, lattice: bool = False):
        mcs, ext = C.c_uint64(), C.c_int32()
        cnt = np.zeros(16, dtype=np.uint64)
        lat = np.empty((self._L[rid], self._L[rid]), dtype=np.uint8) if lattice else None
        check(load().escg_server_result(self._h, int(rid), C.byref(mcs), C.byref(ext),
                                        cnt.ctypes.data_as(C.POINTER(C.c_uint64)),
                                        _u8(lat) if lattice else None))
        return int(mcs.value), bool(ext.value), cnt, lat

    def timing(self, rid: int):
        """(submitted, admitted, finished) host-clock seconds of a finished run
        since the server was created."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        check(load().escg_server_timing(self._h, int(rid), C.byref(a), C.byref(b), C.byref(c)))
        return float(a.value), float(b.value), float(c.value)

    def stats(self):
        r, q, b = C.c_int32(), C.c_int32(), C.c_uint64()
        check(load().escg_server_stats(self._h, C.byref(r), C.byref(q), C.byref(b)))
        return int(r.value), int(q.value), int(b.value)

    @property
    def threads(self) -> int:
        return int(load().escg_server_threads(self._h))

    @property
    def uses_tma(self) -> bool:
        return bool(load().escg_server_uses_tma(self._h))

    @property
    def launches(self) -> int:
        return int(load().escg_server_launch_count(self._h))
