"""Batched-ensemble driver (many independent replicas): runs a list of replica
descriptions in one batch and, for comparison, one run at a time through
the single-lattice path; tabulates extinction per (L, mobility-decade) bin."""
from __future__ import annotations

import math
import time

import numpy as np

from . import Batch, Lattice, circulant
from .serve import request_spec


def run_batch(reps, log_every: int = 10, threads: int = 0, use_graph: bool = True, resident: bool = False) -> dict:
    specs = [request_spec(r) for r in reps]
    t0 = time.perf_counter()
    b = Batch(specs, log_every=log_every, threads=threads, use_graph=use_graph, resident=resident)
    t1 = time.perf_counter()
    b.run()
    mcs, ext, _ = b.status()
    t2 = time.perf_counter()
    site_updates = float(sum(int(m) * s["L"] ** 2 for m, s in zip(mcs, specs)))
    bins = {}
    for r, e in zip(reps, ext):
        key = f"L{r['L']}_M1e{int(math.floor(math.log10(r['mobility'])))}"
        k, n = bins.get(key, (0, 0))
        bins[key] = (k + int(e), n + 1)
    out = {"runs": len(reps), "seconds": t2 - t1, "setup_seconds": t1 - t0,
           "runs_per_s": len(reps) / (t2 - t1), "site_updates_per_s": site_updates / (t2 - t1),
           "threads": b.threads, "staging": "tma" if b.uses_tma else "plain", "launches": b.launches,
           "extinct_fraction": float(np.mean(ext)),
           "extinction_by_bin": {k: round(a / n, 4) for k, (a, n) in sorted(bins.items())},
           "mean_mcs": float(np.mean(mcs))}
    b.close()
    return out, mcs, ext


def run_one_at_a_time(reps, log_every: int = 10) -> dict:
    """The same runs as independent single-lattice runs, one after another
    (per-run launches)."""
    t0 = time.perf_counter()
    mcs = []
    for r in reps:
        sp = request_spec(r)
        g = Lattice(sp["L"], sp["S"], circulant(sp["S"], r["K"]), sp["rates"], sp["seed"],
                    p_empty=sp["p_empty"], log_every=log_every,
                    stop_at_extinction=sp["stop_at_extinction"])
        g.run(sp["max_mcs"])
        mcs.append(g.mcs)
        g.close()
    el = time.perf_counter() - t0
    return {"runs": len(reps), "seconds": el, "runs_per_s": len(reps) / el}, np.array(mcs)
