"""Host-side logic of the serve driver (no GPU): the result ring never hands
out a region that overlaps a request still in flight."""
import random

from paper_1609_00999_gb300.serve import HostRing, latency_summary

import numpy as np


def test_ring_never_overlaps_live_regions():
    rnd = random.Random(3)
    ring = HostRing(1000, 257)
    live = {}
    nxt = 0
    for step in range(20000):
        if live and (rnd.random() < 0.45 or len(live) > 12):
            rid = rnd.choice(sorted(live))
            ring.release(rid)
            del live[rid]
            continue
        n = rnd.randint(1, 90)
        ptr = ring.alloc(nxt, n)
        if ptr is None:
            continue
        s = (ptr - 1000) // 4
        assert 0 <= s and s + n <= 257
        for (a, b) in live.values():
            assert s + n <= a or b <= s, (s, n, a, b)
        live[nxt] = (s, s + n)
        nxt += 1
    assert nxt > 1000


def test_ring_fifo_release_reuses_space():
    ring = HostRing(0, 100)
    assert ring.alloc(0, 60) == 0
    assert ring.alloc(1, 50) is None          # only 40 free
    ring.release(0)
    assert ring.alloc(1, 50) == 0             # empty ring restarts at 0


def test_latency_summary():
    lat = np.array([0.001, 0.002, 0.003, np.nan])
    s = latency_summary(lat)
    assert abs(s["p50_ms"] - 2.0) < 1e-9 and s["max_ms"] == 3.0
