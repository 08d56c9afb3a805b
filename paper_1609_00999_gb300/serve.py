"""Open-loop driver for the request server (``mont_server_*`` in the C ABI).

Requests arrive at given times (a Poisson process in the benchmark); the
driver submits each one when its arrival time has passed, steps the server
with ``progress()``, and records each completion time.  Latency of a request
is completion time minus arrival time, measured on the host clock; the
server does the admission, batching and device work.
"""
import time

import numpy as np

from . import _binding


def run_stream(server, reqs, arrivals, idle_sleep_s=0.0):
    """Drive `server` with requests `reqs` (request_dtype array, ids 0..n-1 in
    order) arriving at `arrivals` seconds (increasing) after the start.

    Returns (latency_s per request, status per request, makespan_s)."""
    n = len(reqs)
    lat = np.full(n, np.nan)
    status = np.zeros(n, dtype=np.int32)
    done = 0
    i = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        j = int(np.searchsorted(arrivals, now, side="right"))
        if j > i:
            server.submit(reqs, i, j)
            i = j
        comps = server.progress()
        if len(comps):
            tc = time.perf_counter() - t0
            ids = comps["id"].astype(np.int64)
            lat[ids] = tc - arrivals[ids]
            status[ids] = comps["status"]
            done += len(comps)
        elif idle_sleep_s:
            time.sleep(idle_sleep_s)
    makespan = time.perf_counter() - t0
    return lat, status, makespan


def make_requests(primes, la, lb, a_ptrs, b_ptrs, c_ptrs):
    """request_dtype array from per-request pointers and sizes."""
    n = len(la)
    reqs = np.zeros(n, dtype=_binding.request_dtype())
    reqs["a"] = a_ptrs
    reqs["b"] = b_ptrs
    reqs["c"] = c_ptrs
    reqs["la"] = la
    reqs["lb"] = lb
    reqs["p"] = primes
    reqs["id"] = np.arange(n, dtype=np.uint64)
    return reqs


def latency_summary(lat):
    lat = lat[np.isfinite(lat)]
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
