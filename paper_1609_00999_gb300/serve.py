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


class HostRing:
    """Result placement in a fixed host buffer of `words` uint32 words.

    Regions are handed out in submission order around the ring; a region is
    reused only after the request holding it (and every older one) has
    completed, so results in flight are never overwritten."""

    def __init__(self, base_ptr, words):
        from collections import deque
        self.base = int(base_ptr)
        self.words = int(words)
        self.head = 0
        self.live = deque()          # [start, end, id, done] in allocation order
        self.by_id = {}

    def alloc(self, rid, n):
        """Word offset region of n words for request rid, as a pointer, or None if full."""
        if n > self.words:
            raise ValueError("result larger than the ring")
        if not self.live:
            start = 0
        else:
            tail = self.live[0][0]                  # oldest region still in use
            if self.head > tail:                    # in use: [tail, head)
                if self.head + n <= self.words:
                    start = self.head
                elif n <= tail:
                    start = 0
                else:
                    return None
            elif self.head + n <= tail:             # in use: [tail, end) and [0, head)
                start = self.head
            else:
                return None
        rec = [start, start + n, rid, False]
        self.live.append(rec)
        self.by_id[rid] = rec
        self.head = start + n
        return self.base + 4 * start

    def release(self, rid):
        rec = self.by_id.pop(rid, None)
        if rec is not None:
            rec[3] = True
        while self.live and self.live[0][3]:
            self.live.popleft()
        if not self.live:
            self.head = 0


def run_stream(server, reqs, arrivals, idle_sleep_s=0.0, ring=None):
    """Drive `server` with requests `reqs` (request_dtype array, ids 0..n-1 in
    order) arriving at `arrivals` seconds (increasing) after the start.  With
    a HostRing, each request's result pointer is assigned from the ring when
    it is submitted (a request whose region is not free yet waits, and its
    latency keeps counting).

    Returns (latency_s per request, status per request, makespan_s)."""
    n = len(reqs)
    lat = np.full(n, np.nan)
    status = np.zeros(n, dtype=np.int32)
    lc = (reqs["la"].astype(np.int64) + reqs["lb"].astype(np.int64) - 1)
    done = 0
    i = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        j = int(np.searchsorted(arrivals, now, side="right"))
        if ring is not None:
            k = i
            while k < j:
                ptr = ring.alloc(k, int(lc[k]))
                if ptr is None:
                    break
                reqs["c"][k] = ptr
                k += 1
            j = k
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
            if ring is not None:
                for rid in ids.tolist():
                    ring.release(rid)
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
