"""Seeded synthetic workloads (inputs only; no modular arithmetic lives here).

This module is the one piece shared by the CUDA path's tests/benchmark and
the CPU oracle's tests: it draws residues, lengths, primes and arrival times
from NumPy's PCG64 generator and nothing else.  The workloads follow the
shapes the paper's setting implies (word-size Fourier primes P = c 2^n + 1,
Sec. 3.1; vectors of residues; polynomial products for the modular FFT
libraries of Sec. 1 and 5):

* elementwise: residues uniform in [0, P), one independent stream per
  (seed, prime index, operand index);
* batched products: coefficient vectors uniform in [0, P);
* uneven batches / request streams: one length L per product (both operands
  have length L), drawn log-uniform in [lo, hi]; prime drawn uniform from the
  three Fourier primes; Poisson arrivals (exponential gaps) for request
  streams.
"""
import concurrent.futures as _cf
import math
import os

import numpy as np

# Fourier primes c 2^n + 1 with 2n >= 32 (Sec. 3.1).
P1 = 2013265921  # 15 * 2^27 + 1
P2 = 469762049   # 7 * 2^26 + 1
P3 = 754974721   # 45 * 2^24 + 1
PRIMES = (P1, P2, P3)

# One base seed per workload.
SEED_ELEMENTWISE_SMALL = 1001   # 65,536 pairs, P1
SEED_ELEMENTWISE_LARGE = 1002   # 2^28 residues per operand, each prime
SEED_BATCH_UNIFORM = 1003       # 4096 products of length 2048, P1
SEED_BATCH_UNEVEN = 1004        # 10,000 products, log-uniform lengths
SEED_SERVE = 1005               # 50,000 Poisson requests


def rng(*key):
    """Independent PCG64 stream for a tuple of non-negative integers."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


_CHUNK = 1 << 22


def _fill_chunk(args):
    out, lo, hi, p, key = args
    out[lo:hi] = rng(*key, lo // _CHUNK).integers(0, p, size=hi - lo, dtype=np.uint32)


def residues(n, p, *key):
    """n residues uniform in [0, p) as uint32.

    Drawn in chunks of 2^22, chunk i from its own stream (key..., i), so the
    values do not depend on how many threads fill the array."""
    out = np.empty(n, dtype=np.uint32)
    jobs = [(out, lo, min(n, lo + _CHUNK), p, key) for lo in range(0, n, _CHUNK)]
    if len(jobs) <= 1:
        for j in jobs:
            _fill_chunk(j)
    else:
        with _cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4, 32)) as ex:
            list(ex.map(_fill_chunk, jobs))
    return out


def loguniform_lengths(count, lo, hi, *key):
    """Lengths L = floor(exp(U(ln lo, ln(hi + 1)))) clamped to [lo, hi]."""
    u = rng(*key).uniform(math.log(lo), math.log(hi + 1), size=count)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), lo, hi)


def choose_primes(count, *key):
    idx = rng(*key).integers(0, len(PRIMES), size=count)
    return np.asarray(PRIMES, dtype=np.uint32)[idx]


def poisson_arrivals(count, rate_per_s, *key):
    """Arrival times (seconds, increasing) of a Poisson process of the given rate."""
    gaps = rng(*key).exponential(1.0 / rate_per_s, size=count)
    return np.cumsum(gaps)


def elementwise_small():
    """65,536 pairs uniform in [0, P1)."""
    n = 65536
    return P1, residues(n, P1, SEED_ELEMENTWISE_SMALL, 0), residues(n, P1, SEED_ELEMENTWISE_SMALL, 1)


def elementwise_large(prime_index, n=1 << 28, operands=3):
    """Operands a, b, c (each n residues uniform in [0, P)) for one of the three primes."""
    p = PRIMES[prime_index]
    return p, [residues(n, p, SEED_ELEMENTWISE_LARGE, prime_index, k) for k in range(operands)]


def batch_uniform(count=4096, length=2048, p=P1):
    """count pairs of length-`length` polynomials, row-major [count][length]."""
    a = residues(count * length, p, SEED_BATCH_UNIFORM, 0).reshape(count, length)
    b = residues(count * length, p, SEED_BATCH_UNIFORM, 1).reshape(count, length)
    return p, a, b


class UnevenBatch:
    """A batch of independent products with per-product prime and length.

    Operands are packed back to back: product i's a occupies
    a[a_off[i] : a_off[i] + la[i]] (likewise b), and its result of length
    la[i] + lb[i] - 1 goes to c[c_off[i] : ...].
    """

    def __init__(self, primes, la, lb, seed_key):
        self.primes = np.asarray(primes, dtype=np.uint32)
        self.la = np.asarray(la, dtype=np.uint64)
        self.lb = np.asarray(lb, dtype=np.uint64)
        n = self.primes.size
        self.a_off = np.zeros(n, dtype=np.uint64)
        self.b_off = np.zeros(n, dtype=np.uint64)
        self.c_off = np.zeros(n, dtype=np.uint64)
        if n:
            self.a_off[1:] = np.cumsum(self.la)[:-1]
            self.b_off[1:] = np.cumsum(self.lb)[:-1]
            self.c_off[1:] = np.cumsum(self.la + self.lb - 1)[:-1]
        self.a_size = int(self.la.sum())
        self.b_size = int(self.lb.sum())
        self.c_size = int((self.la + self.lb - 1).sum()) if n else 0
        # Coefficients uniform in [0, P_i): draw in [0, 2^32) then scale per product.
        g = rng(*seed_key, 7)
        self.a = self._draw(g, self.la, self.a_off, self.a_size)
        self.b = self._draw(g, self.lb, self.b_off, self.b_size)

    def _draw(self, g, lens, offs, size):
        out = np.empty(size, dtype=np.uint32)
        for i in range(self.primes.size):
            o, l = int(offs[i]), int(lens[i])
            out[o:o + l] = g.integers(0, int(self.primes[i]), size=l, dtype=np.uint32)
        return out

    def __len__(self):
        return int(self.primes.size)


def batch_uneven(count=10000, lo=1 << 6, hi=1 << 16, seed=SEED_BATCH_UNEVEN):
    """count products, L log-uniform in [lo, hi], la = lb = L, prime uniform from PRIMES."""
    lens = loguniform_lengths(count, lo, hi, seed, 0)
    primes = choose_primes(count, seed, 1)
    return UnevenBatch(primes, lens, lens, (seed,))


def serve_requests(count=50000, lo=1 << 8, hi=1 << 20, rate_per_s=1000.0, seed=SEED_SERVE):
    """Request stream: (arrival times, UnevenBatch of the requests in arrival order)."""
    lens = loguniform_lengths(count, lo, hi, seed, 0)
    primes = choose_primes(count, seed, 1)
    arrivals = poisson_arrivals(count, rate_per_s, seed, 2)
    return arrivals, UnevenBatch(primes, lens, lens, (seed,))
