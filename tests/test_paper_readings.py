"""CPU checks of the paper's own claims and of the readings taken where the
text is ambiguous (no GPU): Barrett's bound t < 4P before its loop (Sec. 3.1,
Alg. 1) and the validity range of Alg. 3's sign-mask corrections (reading:
exact for Fourier primes below 2^30, wrong for 2013265921)."""
import random

import pytest

from paper_1609_00999_gb300 import synth

R = 1 << 32


def barrett_steps(a, b, p):
    k = (p - 1).bit_length()                    # ceil(log2 p) for p not a power of two
    pb = (1 << (2 * k)) // p
    m = (a * b) >> k
    q = (m * pb) >> k
    t = a * b - q * p
    loops = 0
    while t >= p:
        t -= p
        loops += 1
    return t, loops, a * b - q * p


def to_i32(x):
    x &= 0xFFFFFFFF
    return x - (1 << 32) if x >= (1 << 31) else x


def fourier_redc_printed(a, b, p):
    """Alg. 3 as printed, on 32-bit words with an arithmetic 31-bit shift."""
    w = p - 1                                    # c 2^n
    T = a * b
    q1, r1 = T // R, T % R
    q2, r2 = (w * r1) // R, (w * r1) % R
    q3 = (w * r2) // R
    t = to_i32(q1 - q2 + q3)
    t = to_i32(t + ((t >> 31) & p))
    t = to_i32(t - p)
    t = to_i32(t + ((t >> 31) & p))
    return t & 0xFFFFFFFF


@pytest.mark.parametrize("p", synth.PRIMES)
def test_barrett_bound_and_loop_count(p):
    rnd = random.Random(p)
    vals = [0, 1, p - 1, p - 2, p // 2] + [rnd.randrange(p) for _ in range(20000)]
    worst = 0
    for i in range(len(vals)):
        a, b = vals[i], vals[-1 - i]
        t, loops, t0 = barrett_steps(a, b, p)
        assert t == (a * b) % p
        assert 0 <= t0 < 4 * p and loops <= 3           # the paper's bound
        worst = max(worst, loops)
    assert worst >= 1


@pytest.mark.parametrize("p", [synth.P2, synth.P3, 998244353])
def test_fourier_redc_exact_below_2_30(p):
    rinv = pow(R, -1, p)
    rnd = random.Random(p)
    for _ in range(20000):
        a, b = rnd.randrange(p), rnd.randrange(p)
        assert fourier_redc_printed(a, b, p) == (a * b * rinv) % p


def test_fourier_redc_printed_fails_for_p1():
    p = synth.P1
    rinv = pow(R, -1, p)
    rnd = random.Random(1)
    bad = sum(fourier_redc_printed(a, b, p) != (a * b * rinv) % p
              for a, b in ((rnd.randrange(p), rnd.randrange(p)) for _ in range(20000)))
    assert bad > 0
