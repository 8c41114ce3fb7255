#!/usr/bin/env python3
"""Benchmark of the ESCG Monte Carlo step on GB300.

Metric: site-updates/s (one update = one elementary-step attempt, no-ops
included; N = L^2 per MCS) of a single L = 3200 RPS lattice with empty sites
(S = 3, C(3,{1}), uniform initial states, interaction = reproduction = 1,
exchange = 2 M N with M = 1e-4), counts logged every 10 MCS.  One step =
10 MCS = one log interval, i.e. one pass of every row of the hot path
(coloured-phase lattice update, counts, log).

  value     device time (CUDA events on the library's stream) of K steps,
            L2 flushed (256 MiB write) before every timed step, lattice
            resident in HBM;
  e2e       the same metric through the C ABI with host buffers
            (escg_step_host: pinned host lattice in, K x 10 MCS, lattice and
            counts out, copies inside the timed region);
  roofline  the dominant kernel (the lattice-update kernel the library
            picks, persistent_kernel at L = 3200): algorithmic integer
            instructions per launch / its event-timed launch duration
            against the GPU's integer-issue peak;
  cpu_baseline  the CPU replay oracle (single thread) on a bounded sample;
  ensemble, serving, park, variants, packed  batched runs, a request stream
            to the serving loop, the probabilistic-dominance ensemble and the benchmark
            lattice under the Moore / reflecting rule variants, as
            rectangles of the same N, and the RPSLS L = 800 workload;
            packed: bit-packed lattices (2 bits per site) against one byte per
            site at L = 3200 and 12800; sizes: the same workload at
            L = 128 .. 2560 with the kernel picked for each; each with its
            own metric.

`--impl reference` times the CPU oracle itself (the reference arm of this
tier) on the same metric and workload.  Multi-GPU (torchrun): replicas only,
one independent lattice per rank (weak scaling), max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-updates/s at L=3200 vs roofline; ensemble runs/s and p50/p99 latency"
UNIT = "site-updates/s"

# Algorithmic integer instructions of one elementary step (schedule v1,
# 2x2 sub-blocks): Philox4x32-10 = 10 rounds x (2 wide multiplies + 2
# three-input XORs) per 4 attempts = 10; split of the 32-bit word into
# cell/direction and action draw (1 wide multiply) = 1; cell and neighbour
# tile offsets = 6; two threshold compares and the action select = 3;
# transition-table index = 2; unpacking the new pair = 2; the four
# shared-memory accesses (load a, load b, store a', store b') and the
# table lookup are memory instructions and not counted.
ALG_INT_INSTR_PER_ATTEMPT = 24

# DRAM traffic of persistent_kernel from one ncu capture (bytes per launch of
# a 10-MCS chunk at L = 3200), valid only for that kernel and workload and the
# kernel sources it was taken from (hash below); None otherwise.
NCU_TRAFFIC = {"sources_sha1": "f3d15f12ffa514d9d6328dec9a3d032ff0fde2ee", "bytes_per_launch": 10304768 + 817493,
               "kernel": "persistent_kernel", "L": 3200, "mcs_per_launch": 10,
               "profile": "profiles/persistent_kernel_L3200_M1e-4.md"}


KERNEL_SOURCES = ("escg_kernels.cu", "escg_device.cuh", "escg_types.h", "escg_internal.h", "escg_tma.cuh",
                  "escg_resident.cuh")


def _sources_sha1() -> str:
    """Hash of the translation unit that defines the single-lattice kernels."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2508_16639_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mobility", type=float, default=1e-4)
    ap.add_argument("--mcs-per-step", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-rs-seconds", type=float, default=8.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="time budget of the reference arm's timed steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--persistent", type=int, default=1)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--L", type=int, default=3200, help="lattice side (3200 is the benchmark)")
    ap.add_argument("--neighbourhood", type=int, default=4, choices=[4, 8],
                    help="rule of the main measurement (8: Moore), for profiling the variant builds")
    ap.add_argument("--reflect", action="store_true", help="reflecting boundary for the main measurement")
    ap.add_argument("--workload", choices=["rps", "rpsls-L800"], default="rps",
                    help="rps: the benchmark's RPS lattice (side --L, mobility --mobility); rpsls-L800: the RPSLS "
                         "workload (L = 800, p_empty 0.2, M = 1e-4) for profiling its kernel")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-replicas", type=int, default=1024)
    ap.add_argument("--ensemble-baseline-sample", type=int, default=16)
    ap.add_argument("--ensemble-cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-park", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-sizes", action="store_true")
    ap.add_argument("--no-mobility", action="store_true")
    ap.add_argument("--mobility-steps", type=int, default=200)
    ap.add_argument("--size-steps", type=int, default=100)
    ap.add_argument("--no-packed", action="store_true")
    ap.add_argument("--packed-steps", type=int, default=100)
    ap.add_argument("--variant-steps", type=int, default=100)
    ap.add_argument("--park-per-point", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=200.0,
                    help="mean Poisson arrival rate (requests/s) of the first serving run")
    ap.add_argument("--serve-saturated-requests", type=int, default=4000)
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _workload(M: float, L: int = 3200):
    from paper_2508_16639_gb300 import workloads as W
    import dataclasses
    w = W.CFG3[M] if M in W.CFG3 else dataclasses.replace(W.CFG3[1e-4], name=f"rps-L3200-M{M:g}",
                                                          mobility=M)
    if L != w.L:
        w = dataclasses.replace(w, name=w.name.replace("L3200", f"L{L}"), L=L)
    return w


def _cpu_oracle_rate(w, seconds: float):
    """Replay oracle (single-threaded C) on the seeded initial lattice: whole
    MCS until `seconds` have passed; returns (site-updates/s, MCS done)."""
    import oracle as O
    X = O.exchange_from_mobility(w.mobility, w.L * w.L)
    D = O.circulant(w.S, w.K)
    lat = O.init(w.L, w.S, w.p_empty, w.seed)
    done, t0 = 0, time.perf_counter()
    while True:
        lat, att = O.replay_run(lat, D, w.interact, w.reproduce, X, w.seed, 1, mcs_begin=done)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return done * w.L * w.L / el, done, el


def _hbm_peak():
    """The driver's measured HBM copy bandwidth (MEASURED_PEAKS.json), else
    the profiling recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def _cpu_info():
    """(CPU model, logical cores) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return model, os.cpu_count()


def _cpu_rs_rate(w, seconds: float):
    """Random-sequential oracle (Alg. 3 + Alg. 4, single thread) on the same
    initial lattice: whole MCS until `seconds` have passed."""
    import oracle as O
    X = O.exchange_from_mobility(w.mobility, w.L * w.L)
    D = O.circulant(w.S, w.K)
    lat = O.init(w.L, w.S, w.p_empty, w.seed)
    done, t0 = 0, time.perf_counter()
    while True:
        lat = O.rs_run(lat, D, w.interact, w.reproduce, X, w.seed, 1, mcs_begin=done)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return done * w.L * w.L / el, done, el


def _oracle_ensemble_worker(job):
    """One host core: the schedule-v1 replay oracle on its share of the
    ensemble's replicas, in order, each to extinction or its budget in
    chunks of 10 MCS, until `seconds` have passed.  Returns (site-updates,
    runs finished, seconds)."""
    reps, seconds = job
    import oracle as O
    t0 = time.perf_counter()
    upd, fin = 0, 0
    for r in reps:
        L, S = r["L"], r["S"]
        X = O.exchange_from_mobility(r["mobility"], L * L)
        D = O.circulant(S, r["K"])
        lat = O.init(L, S, r["p_empty"], r["seed"])
        m, finished = 0, False
        while not finished:
            n = min(10, r["max_mcs"] - m)
            lat, _, mend = O.run_observed(lat, D, r["interact"], r["reproduce"], X, r["seed"], n, log_every=10,
                                          stop_at_extinction=True, mcs_begin=m)
            upd += (mend - m) * L * L
            finished = mend < m + n or mend >= r["max_mcs"]
            m = mend
            if time.perf_counter() - t0 >= seconds:
                break
        fin += int(finished)
        if time.perf_counter() - t0 >= seconds:
            break
    return upd, fin, time.perf_counter() - t0


def _oracle_ensemble_rate(reps, seconds: float, mean_updates_per_run: float):
    """The ensemble on every host core: one oracle process per core (spawned,
    so that no CUDA state is inherited), replicas dealt round-robin, a
    bounded wall time.  Runs/s = aggregate site-updates/s divided by the
    mean site-updates of a run of this ensemble (from the GPU run, whose
    runs are the same)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [(reps[k::cores], seconds) for k in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_ensemble_worker, jobs)
    wall = time.perf_counter() - t0
    upd = sum(r[0] for r in res)
    fin = sum(r[1] for r in res)
    rate = upd / max(r[2] for r in res)
    return {"value": rate / mean_updates_per_run, "unit": "runs/s", "cores": cores, "kind": "oracle",
            "site_updates_per_s": rate, "runs_finished_in_sample": fin, "wall_s": wall,
            "sample": f"schedule-v1 replay oracle, one process per core over the ensemble's replicas "
                      f"(round-robin), {seconds:g} s each; runs/s = site-updates/s / mean site-updates of "
                      f"a run ({mean_updates_per_run:.3g})"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    w = _workload(args.mobility)
    X = O.exchange_from_mobility(w.mobility, w.L * w.L)
    D = O.circulant(w.S, w.K)
    lat = O.init(w.L, w.S, w.p_empty, w.seed)
    m = 0
    for _ in range(min(args.warmup, 3)):
        lat, _ = O.replay_run(lat, D, w.interact, w.reproduce, X, w.seed, 1, mcs_begin=m)
        m += 1
    # One step = one MCS of the benchmark lattice (about 0.35 s on one core):
    # the timed steps stop after --ref-seconds, so that the run stays within
    # a few minutes whatever --steps asks for; the line reports the steps
    # actually timed.
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        lat, _ = O.replay_run(lat, D, w.interact, w.reproduce, X, w.seed, 1, mcs_begin=m)
        m += 1
        done += 1
        if time.perf_counter() - t0 >= args.ref_seconds:
            break
    el = time.perf_counter() - t0
    value = done * w.L * w.L / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": done, "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": _config(w, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"schedule-v1 replay oracle, 1 MCS of the L={w.L} lattice per step, "
                                   f"{done} steps timed (at most {args.ref_seconds:g} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(w, mcs_per_step):
    return {"workload": w.name, "L": w.L, "S": w.S, "digraph": f"C({w.S},{set(w.K)})",
            "mobility": w.mobility, "p_empty": w.p_empty, "interact": w.interact,
            "reproduce": w.reproduce, "mcs_per_step": mcs_per_step, "log_every": w.log_every,
            "l2": f"flushed before every timed step (256 MiB write); lattice {w.L * w.L / 1e6:.2f} MB",
            "parallelism": "replicas (one independent lattice per GPU)"}


def _ensemble(args, rank, world, dist):
    """Batched ensemble: independent replicas (L uniform on {64,100,200,400},
    RPS/RPSLS, M log-uniform on [1e-5, 1e-3]) each to extinction or 10^4 MCS
    in shared persistent launches, the replicas dealt round-robin over the
    ranks; beside it, a sample of the same runs as per-run launches (one
    single-lattice handle per run, each on its own stream, all in flight at
    once) and the CPU oracle on every host core."""
    import numpy as np
    import torch
    from paper_2508_16639_gb300 import Lattice, circulant, replicas as R
    from paper_2508_16639_gb300 import workloads as W
    from paper_2508_16639_gb300.ensemble import run_batch
    from paper_2508_16639_gb300.serve import request_spec
    reps_all = W.ensemble(args.ensemble_replicas, seed=1)
    reps = R.shard(reps_all, rank, world)
    if dist is not None:
        dist.barrier()
    out, mcs, ext = run_batch(reps)
    secs = R.max_over_ranks(out["seconds"], dist, device="cuda")
    out["runs"] = len(reps_all)
    out["runs_per_s"] = len(reps_all) / secs
    out["site_updates_per_s"] = R.sum_over_ranks(out["site_updates_per_s"] * out["seconds"], dist,
                                                 device="cuda") / secs
    out["seconds"] = secs
    # per-run launches: the sample's runs as concurrent single-lattice handles
    sample_idx = np.random.default_rng(0).choice(len(reps), min(args.ensemble_baseline_sample, len(reps)),
                                                 replace=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs = []
    for i in sample_idx:
        sp = request_spec(reps[i])
        g = Lattice(sp["L"], sp["S"], circulant(sp["S"], reps[i]["K"]), sp["rates"], sp["seed"],
                    p_empty=sp["p_empty"], log_every=10, stop_at_extinction=sp["stop_at_extinction"],
                    stream=torch.cuda.Stream())
        g.run(sp["max_mcs"])
        hs.append(g)
    for g in hs:
        g.sync()
    el = time.perf_counter() - t0
    mcs1 = np.array([g.mcs for g in hs])
    for g in hs:
        g.close()
    base = {"runs": len(sample_idx), "seconds": el, "runs_per_s": len(sample_idx) / el,
            "sample": f"{len(sample_idx)} of the same runs, one single-lattice handle per run, each on its own "
                      "stream, all enqueued before the first is waited for (creation included)",
            "identical_mcs": bool(np.array_equal(mcs1, mcs[sample_idx]))}
    out["per_run_launches"] = base
    out["speedup_vs_per_run"] = out["runs_per_s"] / world / base["runs_per_s"]   # per GPU
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_run = out["site_updates_per_s"] * secs / len(reps_all)
        out["cpu_baseline"] = _oracle_ensemble_rate(reps_all, args.ensemble_cpu_seconds, per_run)
    out["metric"] = "ensemble runs/s"
    out["config"] = {"workload": f"{len(reps_all)} replicas, L in {{64,100,200,400}}, S in {{3,5}}, "
                                 "M log-uniform [1e-5,1e-3], to extinction or 10^4 MCS, log every 10 MCS",
                     "ranks": world, "split": "round-robin over ranks (replicas.shard)"}
    return out


def _park(args, rank, world, dist):
    """Probabilistic-dominance ensemble (the Park, Chen and Szolnoki model the
    paper replicates): L = 100, 8 species, edge probabilities (alpha, beta,
    gamma = 1), no mobility, L^2 MCS or until one species is left; reports
    runs/s and the distribution of surviving species per (alpha, beta)."""
    import time
    import numpy as np
    from paper_2508_16639_gb300 import workloads as W
    from paper_2508_16639_gb300 import Batch
    from paper_2508_16639_gb300 import replicas as R
    specs_all = W.park_ensemble(per_point=args.park_per_point)
    specs = R.shard(specs_all, rank, world)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    b = Batch([{k: v for k, v in sp.items() if k != "point"} for sp in specs], log_every=10)
    t1 = time.perf_counter()
    b.run()
    mcs, ext, cnt = b.status()
    t2 = time.perf_counter()
    surv = {}
    for sp, c in zip(specs, cnt):
        key = "a%.1f_b%.1f" % sp["point"]
        n = int((c[1:9] > 0).sum())
        surv.setdefault(key, np.zeros(9, dtype=int))[n] += 1
    site_updates = float(sum(int(m) * sp["L"] ** 2 for m, sp in zip(mcs, specs)))
    secs = R.max_over_ranks(t2 - t1, dist, device="cuda")
    out = {"metric": "probabilistic-dominance ensemble runs/s", "runs": len(specs_all),
           "seconds": secs, "setup_seconds": t1 - t0, "runs_per_s": len(specs_all) / secs,
           "site_updates_per_s": R.sum_over_ranks(site_updates, dist, device="cuda") / secs,
           "threads": b.threads, "staging": "tma" if b.uses_tma else "plain", "launches": b.launches,
           "mean_mcs": float(np.mean(mcs)),
           "surviving_species_histogram": {k: v.tolist() for k, v in sorted(surv.items())},
           "config": {"workload": f"{len(specs_all)} replicas: L=100, 8 species beating the next 3 with "
                                  "probabilities (alpha, beta, 1), alpha, beta in {0.2,0.5,0.8}, "
                                  "I=P=1, no mobility, to one species or L^2 MCS"}}
    b.close()
    return out


def _variants(args, rank, w):
    """The benchmark lattice under the paper's rule variants (Moore
    neighbourhood, reflecting boundary), as rectangles of the same N
    (2L x L/2 and L/2 x 2L), and the RPSLS L = 800 workload (generic
    partition: 12 blocks of 66-67 sites per axis): device time per 10-MCS
    step, L2 flushed before each step, as the main measurement."""
    import torch
    import paper_2508_16639_gb300 as E
    from paper_2508_16639_gb300 import replicas as R
    from paper_2508_16639_gb300 import workloads as W
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    c2 = W.CFG2
    cases = [("moore", w, w.L, w.L, 8, False), ("reflect", w, w.L, w.L, 4, True),
             ("moore_reflect", w, w.L, w.L, 8, True),
             (f"rect_{2 * w.L}x{w.L // 2}", w, 2 * w.L, w.L // 2, 4, False),
             (f"rect_{w.L // 2}x{2 * w.L}", w, w.L // 2, 2 * w.L, 4, False),
             (c2.name, c2, c2.L, c2.L, 4, False)]
    for name, wl, Lc, Hr, nbh, refl in cases:
        N = Lc * Hr
        X = E.exchange_from_mobility(wl.mobility, N)
        stream = torch.cuda.Stream()
        g = E.Lattice(Lc, wl.S, E.circulant(wl.S, wl.K), (wl.interact, wl.reproduce, X),
                      R.replica_seed(wl.seed, rank), p_empty=wl.p_empty, log_every=wl.log_every, stream=stream,
                      neighbourhood=nbh, reflecting_boundary=refl, H=Hr)
        for _ in range(3):
            g.run(10)
        g.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.variant_steps)]
        for a, b in ev:
            with torch.cuda.stream(stream):
                flush.fill_(1)
            a.record(stream)
            g.run(10)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        out[name] = {"site_updates_per_s": 10 * N / (ms * 1e-3), "ms_per_10_mcs": ms,
                     "kernel": g.update_kernel}
        g.close()
    out["config"] = {"workload": f"{w.name} with the Moore neighbourhood and/or a reflecting boundary; "
                                 "rect_<columns>x<rows>: the same N = L*L as a rectangle; "
                                 f"{c2.name}: S=5 C(5,{{1,2}}), p_empty {c2.p_empty}, M {c2.mobility:g}",
                     "steps": args.variant_steps}
    return out


def _mobility_points(args, rank, w):
    """The benchmark lattice (L = 3200, RPS with empty sites) at the other two
    mobilities of the workload, M = 1e-5 and 1e-3 (exchange 2MN: 99.0 % and
    99.9 % of attempts), timed as the main measurement: device time per 10-MCS
    step, L2 flushed before each step."""
    import torch
    import paper_2508_16639_gb300 as E
    from paper_2508_16639_gb300 import replicas as R
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for M in (1e-5, 1e-3):
        wm = _workload(M, w.L)
        N = wm.L * wm.L
        X = E.exchange_from_mobility(M, N)
        stream = torch.cuda.Stream()
        g = E.Lattice(wm.L, wm.S, E.circulant(wm.S, wm.K), (wm.interact, wm.reproduce, X),
                      R.replica_seed(wm.seed, rank), p_empty=wm.p_empty, log_every=wm.log_every, stream=stream,
                      time_kernels=True)
        for _ in range(3):
            g.run(10)
        g.sync()
        g.kernel_time(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.mobility_steps)]
        for a, b in ev:
            with torch.cuda.stream(stream):
                flush.fill_(1)
            a.record(stream)
            g.run(10)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        kms, kn = g.kernel_time()
        out[wm.name] = {"site_updates_per_s": 10 * N / (ms * 1e-3), "ms_per_10_mcs": ms,
                        "kernel_ms_per_launch": kms / max(1, kn), "exchange": X, "kernel": g.update_kernel}
        g.close()
    out["config"] = {"workload": f"{w.name} at M = 1e-5 and 1e-3", "steps": args.mobility_steps}
    return out


def _sizes(args, rank, w):
    """Latency-bound and mid sizes: the benchmark's workload (RPS with empty
    sites, M = 1e-4) on L x L lattices from 128 to 3200 (uniform and generic
    partitions), each timed with every fixed launch mode (flag 3, TMA 2,
    block owners 5, mailbox 6), the default size rule (1) and the
    autotuner's choice (1 with autotune): device time per 10-MCS step, L2
    flushed before each step.  tuned_vs_best: the tuned time over the best
    fixed mode's."""
    import torch
    import paper_2508_16639_gb300 as E
    from paper_2508_16639_gb300 import replicas as R
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(Lc, **kw):
        N = Lc * Lc
        X = E.exchange_from_mobility(w.mobility, N)
        stream = torch.cuda.Stream()
        g = E.Lattice(Lc, w.S, E.circulant(w.S, w.K), (w.interact, w.reproduce, X), R.replica_seed(w.seed, rank),
                      p_empty=w.p_empty, log_every=w.log_every, stream=stream, **kw)
        for _ in range(3):
            g.run(10)
        g.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.size_steps)]
        for a, b in ev:
            with torch.cuda.stream(stream):
                flush.fill_(1)
            a.record(stream)
            g.run(10)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        res = {"us_per_mcs": ms * 100.0, "site_updates_per_s": 10 * N / (ms * 1e-3), "kernel": g.update_kernel}
        if kw.get("autotune"):
            mode, ctas, _, n = g.autotune_result
            res.update(mode=mode, ctas_per_sm=ctas, configurations_timed=n)
        g.close()
        return res

    out = {}
    for Lc in (128, 512, 800, 1024, 1536, 2048, 2200, 2560, 3200):
        fixed = {f"mode{m}": timed(Lc, persistent=m) for m in (3, 2, 5, 6)}
        best = min(v["us_per_mcs"] for v in fixed.values())
        default = timed(Lc)
        tuned = timed(Lc, autotune=True)
        out[f"L{Lc}"] = {"default": default, "tuned": tuned, "fixed": fixed,
                         "tuned_vs_best": tuned["us_per_mcs"] / best,
                         "default_vs_best": default["us_per_mcs"] / best,
                         # the headline's own fields: the default choice
                         "us_per_mcs": default["us_per_mcs"], "kernel": default["kernel"]}
    out["config"] = {"workload": f"{w.name} workload on L x L lattices; modes that a lattice cannot run fall back "
                                 "to the flag kernel", "steps": args.size_steps}
    return out


def _packed(args, rank, w):
    """Bit-packed device lattices: the benchmark lattice and one 4x larger
    (L = 12800: 164 MB with one byte per site, more than the 129 MB L2; 41 MB
    with 2 bits per site) with 8 and 2 bits per site, device time per 10-MCS
    step, L2 flushed before each step."""
    import torch
    import paper_2508_16639_gb300 as E
    from paper_2508_16639_gb300 import replicas as R
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for L, steps in ((w.L, args.packed_steps), (4 * w.L, max(3, args.packed_steps // 8))):
        N = L * L
        X = E.exchange_from_mobility(w.mobility, N)
        for bits in (8, 2):
            stream = torch.cuda.Stream()
            g = E.Lattice(L, w.S, E.circulant(w.S, w.K), (w.interact, w.reproduce, X),
                          R.replica_seed(w.seed, rank), p_empty=w.p_empty, log_every=w.log_every, stream=stream,
                          bits_per_site=bits)
            for _ in range(3):
                g.run(10)
            g.sync()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            for a, b in ev:
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                a.record(stream)
                g.run(10)
                b.record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
            out[f"L{L}_bits{bits}"] = {"site_updates_per_s": 10 * N / (ms * 1e-3), "ms_per_10_mcs": ms,
                                       "device_bytes": E.lattice_bytes(L, L, bits), "kernel": g.update_kernel,
                                       "steps": steps}
            g.close()
    out["config"] = {"workload": f"{w.name} and the same rates at 4x the side, 8 and 2 bits per site"}
    return out


def _serve_shard(args, rank, world, dist, rate, n):
    """One request stream at mean rate `rate` (requests/s over all ranks),
    its requests dealt round-robin over the ranks; runs/s over all ranks and
    latency percentiles over every request."""
    import numpy as np
    from paper_2508_16639_gb300 import replicas as R
    from paper_2508_16639_gb300 import workloads as W
    from paper_2508_16639_gb300.serve import serve
    reqs = R.shard(W.request_stream(n=n, seed=2, rate_per_s=rate), rank, world)
    if dist is not None:
        dist.barrier()
    out = serve(reqs, arena_bytes=4 << 30, max_slots=4096, chunks_per_step=4)
    lat = np.asarray(out.pop("latencies_s"))
    secs = R.max_over_ranks(out["seconds"], dist, device="cuda")
    if dist is not None:
        parts = [None] * world
        dist.all_gather_object(parts, lat.tolist())
        lat = np.concatenate([np.asarray(p) for p in parts])
    out.update(runs=int(lat.size), seconds=secs, runs_per_s=lat.size / secs,
               p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
               mean_latency_s=float(lat.mean()), offered_rate_per_s=rate)
    return out


def _serving(args, rank, world, dist):
    """Serving: Poisson arrivals of run requests (L log-uniform [50,1600],
    S in {3,5}, budgets log-uniform 10^2-10^4 MCS, half stop at extinction),
    continuous batching with admission by free device memory; at the default
    offered rate and at twice the rate the first run sustained (above
    capacity: the queue grows, and runs/s is the capacity)."""
    out = _serve_shard(args, rank, world, dist, args.serve_rate, args.serve_requests)
    sat_rate = 2.0 * out["runs_per_s"]
    out["saturated"] = _serve_shard(args, rank, world, dist, sat_rate, args.serve_saturated_requests)
    out["metric"] = "served runs/s and p50/p99 latency (arrival to result)"
    out["config"] = {"workload": f"{args.serve_requests} requests, Poisson rate {args.serve_rate}/s "
                                 f"(saturated: {args.serve_saturated_requests} requests at twice the sustained "
                                 "runs/s), L log-uniform [50,1600], S in {3,5}, budget log-uniform [1e2,1e4] MCS, "
                                 "50% stop at extinction", "arena_bytes": 4 << 30, "max_slots": 4096,
                     "ranks": world, "split": "round-robin over ranks (replicas.shard)"}
    return out


def main():
    args = _parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    from paper_2508_16639_gb300 import replicas as R
    rank, world, local = R.rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import paper_2508_16639_gb300 as E

    if args.workload == "rpsls-L800":
        from paper_2508_16639_gb300 import workloads as W
        w = W.CFG2
    else:
        w = _workload(args.mobility, args.L)
    N = w.L * w.L
    X = E.exchange_from_mobility(w.mobility, N)
    stream = torch.cuda.Stream()
    g = E.Lattice(w.L, w.S, E.circulant(w.S, w.K), (w.interact, w.reproduce, X), R.replica_seed(w.seed, rank),
                  p_empty=w.p_empty, log_every=w.log_every, stream=stream, time_kernels=True,
                  persistent=args.persistent, ctas_per_sm=args.ctas_per_sm, neighbourhood=args.neighbourhood,
                  reflecting_boundary=args.reflect)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, Wm, mps = args.steps, args.warmup, args.mcs_per_step

    for _ in range(Wm):
        g.run(mps)
    g.sync()
    g.kernel_time(reset=True)
    launches0 = g.launches
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        starts[k].record(stream)
        g.run(mps)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    g.sync()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    kernel_ms, kernel_n = g.kernel_time()
    gpu_launches = g.launches - launches0
    ms = R.max_over_ranks(ms, dist, device="cuda")
    attempts = K * mps * N * world
    value = attempts / (ms * 1e-3)

    # roofline of the dominant kernel.  Integer issue binds (the lattice is
    # L2-resident): achieved = the 24 algorithmic integer instructions of an
    # attempt x attempts per launch / the launch's event-timed duration;
    # peak = the measured throughput of a probe running exactly that
    # instruction mix (escg_diag_alg_throughput) per SM per clock x SMs x the
    # maximum SM clock.  Bandwidth, as a second view: the algorithmic tile
    # traffic (2 B per attempt) against the measured L2-resident copy
    # bandwidth and the driver's measured HBM copy bandwidth.
    alg_s, alg_sm_clk = E.alg_throughput()
    ops_s, ops_sm_clk = E.int_throughput()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    sm_max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * alg_sm_clk * sm_max_mhz * 1e6  # instructions of the step's mix per second
    per_launch_attempts = mps * N  # one persistent launch = one 10-MCS chunk
    avg_launch_s = (kernel_ms * 1e-3) / max(1, kernel_n)
    achieved = per_launch_attempts * ALG_INT_INSTR_PER_ATTEMPT / avg_launch_s
    traffic = (NCU_TRAFFIC["bytes_per_launch"]
               if (NCU_TRAFFIC["sources_sha1"] == _sources_sha1() and g.update_kernel == NCU_TRAFFIC["kernel"]
                   and w.L == NCU_TRAFFIC["L"] and mps == NCU_TRAFFIC["mcs_per_launch"]) else None)
    tile_gbs = 2.0 * per_launch_attempts / avg_launch_s / 1e9
    l2_peak = E.l2_copy_gbs(N, 200)
    hbm_peak, hbm_src = _hbm_peak()
    roofline = {"bound": "alu", "kernel": g.update_kernel,
                "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tinstr/s",
                "frac": achieved / peak, "traffic": traffic,
                "alg_int_instr_per_attempt": ALG_INT_INSTR_PER_ATTEMPT,
                "attempts_per_launch": per_launch_attempts,
                "avg_launch_ms": avg_launch_s * 1e3, "launches_timed": kernel_n,
                "peak_derivation": f"{sms} SMs x {alg_sm_clk:.1f} instructions of the step's mix per SM per clock "
                                   f"(measured probe) x {sm_max_mhz:.0f} MHz",
                "probe_alg_instr_per_s": alg_s, "probe_alg_instr_per_sm_clk": alg_sm_clk,
                "probe_philox_pair_instr_per_sm_clk": ops_sm_clk,
                "issue_ceiling": {"peak": sms * 128 * sm_max_mhz * 1e6 / 1e12, "unit": "Tinstr/s",
                                  "frac_alg": achieved / (sms * 128 * sm_max_mhz * 1e6),
                                  "note": "4 schedulers x 32 lanes per SM per clock; algorithmic instructions"},
                "l2": {"achieved_gbs": tile_gbs, "peak_gbs": l2_peak, "frac": tile_gbs / l2_peak,
                       "peak_source": f"measured: copy between two L2-resident {N / 1e6:.2f} MB buffers"},
                "hbm": {"achieved_gbs": tile_gbs, "peak_gbs": hbm_peak, "frac": tile_gbs / hbm_peak,
                        "peak_source": hbm_src}}

    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(g.snapshot()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        a, b = host_in.numpy(), host_out.numpy()
        m0 = g.mcs
        g.step_host(a, m0, mps, out=b)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            g.step_host(a, m0, mps, out=b)
        el_sync = time.perf_counter() - t0
        el_sync = R.max_over_ranks(el_sync, dist, device="cuda")
        # Pipelined: two handles used alternately with the asynchronous call,
        # so that one step's copies overlap the other's kernel; every step
        # still copies its lattice in and its lattice and counts out.
        g2 = E.Lattice(w.L, w.S, E.circulant(w.S, w.K), (w.interact, w.reproduce, X),
                       R.replica_seed(w.seed, rank), p_empty=w.p_empty, log_every=w.log_every,
                       stream=torch.cuda.Stream())
        hs = (g, g2)
        outs = [torch.empty_like(host_in).pin_memory().numpy() for _ in hs]
        cnts = [torch.zeros(w.S + 1, dtype=torch.int64).pin_memory().numpy().view(np.uint64) for _ in hs]
        for i, h in enumerate(hs):   # warm
            h.step_host_async(a, m0, mps, outs[i], cnts[i])
            h.step_host_wait()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            i = k & 1
            if k >= 2:
                hs[i].step_host_wait()
            hs[i].step_host_async(a, m0, mps, outs[i], cnts[i])
        for k in range(max(0, K - 2), K):
            hs[k & 1].step_host_wait()
        el = time.perf_counter() - t0
        el = R.max_over_ranks(el, dist, device="cuda")
        assert np.array_equal(outs[0], b) and np.array_equal(outs[1], b)   # same step, same result
        g2.close()
        e2e = {"value": K * mps * N * world / el, "unit": UNIT, "h2d_bytes_per_step": N,
               "d2h_bytes_per_step": N + 8 * (w.S + 1), "ms_per_step": 1e3 * el / K,
               "api": "escg_step_host_async + escg_step_host_wait on two handles used alternately "
                      "(each step: pinned lattice in, 10 MCS, lattice and counts out)",
               "sync": {"value": K * mps * N * world / el_sync, "ms_per_step": 1e3 * el_sync / K,
                        "api": "escg_step_host on one handle (restore + run + snapshot + counts)"}}

    mobility = None
    if not args.no_mobility:
        mobility = _mobility_points(args, rank, w)
    packed = None
    if not args.no_packed:
        packed = _packed(args, rank, w)
    variants = None
    if not args.no_variants:
        variants = _variants(args, rank, w)
    sizes = None
    if not args.no_sizes:
        sizes = _sizes(args, rank, w)
    ensemble = None
    if not args.no_ensemble:
        ensemble = _ensemble(args, rank, world, dist)
    serving = None
    if not args.no_serving:
        serving = _serving(args, rank, world, dist)
    park = None
    if not args.no_park:
        park = _park(args, rank, world, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nmcs, el = _cpu_oracle_rate(w, args.cpu_seconds)
        rs_rate, rs_mcs, rs_el = _cpu_rs_rate(w, args.cpu_rs_seconds)
        model, ncpu = _cpu_info()
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"schedule-v1 replay oracle, first {nmcs} MCS of the L={w.L} lattice "
                         f"({el:.1f} s, single thread)",
               "cpu_model": model, "nproc": ncpu,
               "random_sequential": {"value": rs_rate, "unit": UNIT, "cores": 1,
                                     "sample": f"random-sequential oracle (Alg. 3 + Alg. 4), first {rs_mcs} MCS "
                                               f"of the same lattice ({rs_el:.1f} s, single thread)"}}

    if rank == 0:
        # the sections with their own metrics last (ensemble, serving, park)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": _config(w, mps), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": gpu_launches, "clocks": clocks,
                "context": {"paper_cuda_ms_L3200_site_updates_per_s": 2.45e8,
                            "paper_hardware": "RTX A2000 (not a target)"},
                "mobility": mobility, "variants": variants, "packed": packed, "sizes": sizes,
                "ensemble": ensemble, "serving": serving, "park": park}
        if args.neighbourhood != 4 or args.reflect:
            line["config"].update(neighbourhood=args.neighbourhood, reflecting_boundary=bool(args.reflect))
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
