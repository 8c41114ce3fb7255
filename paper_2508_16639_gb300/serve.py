"""Request loop over the continuous-batching server (runs arriving over time).

`serve()` replays a stream of run requests in real time: each request is
submitted to the server when its (scaled) arrival time has passed, the
server is stepped while it holds work, and a request's latency is measured
from its arrival to the step that retires it, split into the wait in the
queue and the time in service (escg_server_timing).  The loop itself is host-side
orchestration; admission, execution and retirement happen in libescg.
"""
from __future__ import annotations

import time

import numpy as np

from . import Server, circulant, exchange_from_mobility


def request_spec(req) -> dict:
    """Turns a request description (L, S, K, mobility, ...) into a run spec."""
    L, S = int(req["L"]), int(req["S"])
    X = exchange_from_mobility(req["mobility"], L * L) if req.get("mobility") is not None else \
        float(req.get("exchange", 0.0))
    return dict(L=L, S=S, digraph=circulant(S, req["K"]), rates=(req["interact"], req["reproduce"], X),
                seed=req["seed"], p_empty=req["p_empty"], max_mcs=req["max_mcs"],
                stop_at_extinction=req["stop_at_extinction"])


def serve(requests, server: Server | None = None, time_scale: float = 1.0, **server_kwargs) -> dict:
    srv = server if server is not None else Server(**server_kwargs)
    order = sorted(range(len(requests)), key=lambda i: requests[i]["arrival_s"])
    arrival = {}
    latency = {}
    done_mcs = {}
    parts = {}   # request -> (queue wait, in service), seconds on the server's clock
    nxt = 0
    n = len(requests)
    steps = 0
    t0 = time.perf_counter()
    while len(latency) < n:
        now = time.perf_counter() - t0
        while nxt < n and requests[order[nxt]]["arrival_s"] * time_scale <= now:
            i = order[nxt]
            rid = srv.submit(request_spec(requests[i]))
            arrival[rid] = (i, requests[i]["arrival_s"] * time_scale)
            nxt += 1
        resident, queued, _ = srv.stats()
        if resident + queued > 0:
            srv.step()
            steps += 1
        elif nxt < n:
            time.sleep(max(0.0, requests[order[nxt]]["arrival_s"] * time_scale
                           - (time.perf_counter() - t0)))
        t_done = time.perf_counter() - t0
        for rid in srv.poll():
            i, t_arr = arrival[rid]
            latency[i] = t_done - t_arr
            done_mcs[i] = srv.result(rid)[0]
            t_sub, t_adm, t_fin = srv.timing(rid)
            parts[i] = (t_adm - t_sub, t_fin - t_adm)
    total = time.perf_counter() - t0
    lat = np.array([latency[i] for i in range(n)])
    pr = np.array([parts[i] for i in range(n)])
    breakdown = {f"{name}_{q}_s": float(np.percentile(pr[:, k], p))
                 for k, name in enumerate(("queue", "service")) for q, p in (("p50", 50), ("p99", 99))}
    return {"runs": n, "seconds": total, "runs_per_s": n / total, "steps": steps,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "latencies_s": lat.tolist(),
            "site_updates": float(sum(done_mcs[i] * requests[i]["L"] ** 2 for i in range(n))),
            "threads": srv.threads, "staging": "tma" if srv.uses_tma else "plain",
            # arrival to result = (at most one step until submission) + queue
            # wait (submission to admission) + service (admission to the step
            # that retires the run)
            "latency_breakdown": breakdown}
