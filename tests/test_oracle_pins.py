"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics.

The oracle computes everything from definitions with 64-bit `%`; these tests
check it against things other than itself: hand-derived closed forms and
worked examples (tests/golden), the integer identity R R^-1 - P P' = 1 and the
REDC identity (Sec. 3.1), brute force over all pairs for tiny moduli, an
independent pure-Python REDC written from Alg. 2, Fermat's little theorem,
the order of the roots of unity, closed-form DFTs, Horner evaluation, the
convolution theorem and exact big-integer (Kronecker) polynomial products.
"""
import os
import random

import numpy as np
import pytest

import oracle
from paper_1609_00999_gb300 import synth

R = 1 << 32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY_ODD = [3, 5, 7, 9, 15, 17, 97, 255, 257]
TINY_PRIMES = [3, 5, 7, 17, 97, 257, 7681, 12289]


def _golden_constants():
    rows = []
    with open(os.path.join(GOLDEN, "prime_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p, c, n, rmodp, pprime, rinv, g, fac = line.split()
            rows.append(dict(p=int(p), c=int(c), n=int(n), rmodp=int(rmodp), pprime=int(pprime),
                             rinv=int(rinv), g=int(g), factors=fac))
    return rows


def _golden_examples():
    out = []
    with open(os.path.join(GOLDEN, "small_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("->")
            parts = lhs.split()
            out.append((parts[0], int(parts[1]), parts[2:], [int(v) for v in rhs.split(",")]))
    return out


def _parse_factors(s):
    fac = {}
    for term in s.split("*"):
        if "^" in term:
            b, e = term.split("^")
            fac[int(b)] = int(e)
        else:
            fac[int(term)] = 1
    return fac


# ---------------------------------------------------------------- Sec. 3.1 constants

@pytest.mark.parametrize("row", _golden_constants(), ids=lambda r: str(r["p"]))
def test_setup_matches_closed_forms(row):
    p = row["p"]
    assert p == row["c"] * 2 ** row["n"] + 1 and 2 * row["n"] >= 32
    c = oracle.setup(p)
    assert c.p_prime == row["pprime"] == p - 2
    assert c.r_inv == row["rinv"]
    assert c.r_mod_p == row["rmodp"]
    # R R^-1 - P P' = 1 as an integer identity, with the stated ranges.
    assert R * c.r_inv - p * c.p_prime == 1
    assert 0 < c.r_inv < p and 0 < c.p_prime < R
    # R^2 mod P is pinned through R^-1: (R^2 mod P) R^-1 R^-1 == 1 (mod P).
    assert c.r2_mod_p < p and (c.r2_mod_p * c.r_inv * c.r_inv) % p == 1


@pytest.mark.parametrize("p", TINY_ODD + [2 ** 31 - 1, 1000000007 % (2 ** 31), 65537])
def test_setup_identity_any_odd_modulus(p):
    c = oracle.setup(p)
    assert R * c.r_inv - p * c.p_prime == 1
    assert 0 < c.r_inv < p and 0 < c.p_prime < R
    assert (p * c.p_prime) % R == R - 1          # P' = -P^-1 mod R


@pytest.mark.parametrize("p", [0, 1, 2, 4, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 1])
def test_setup_rejects_bad_moduli(p):
    with pytest.raises(ValueError):
        oracle.setup(p)


# ---------------------------------------------------------------- REDC semantics

def _redc_alg2(a, b, p, pprime):
    """Alg. 2 written out with Python integers (independent of the oracle's R^-1 route)."""
    T = a * b
    m = ((T % R) * pprime) % R
    t = (T + m * p) // R
    assert (T + m * p) % R == 0 and 0 <= t < 2 * p
    return t - p if t >= p else t


@pytest.mark.parametrize("p", TINY_ODD)
def test_mont_mul_brute_force_all_pairs(p):
    """For every pair, z = REDC(x, y) satisfies z R == x y (mod P), 0 <= z < P (Sec. 3.1)."""
    xs = np.repeat(np.arange(p, dtype=np.uint32), p)
    ys = np.tile(np.arange(p, dtype=np.uint32), p)
    z = oracle.mont_mul(p, xs, ys).astype(np.int64)
    assert np.all(z < p)
    assert np.all((z * (R % p) - xs.astype(np.int64) * ys) % p == 0)
    c = oracle.setup(p)
    for x, y, zz in zip(xs.tolist(), ys.tolist(), z.tolist()):
        assert zz == _redc_alg2(x, y, p, c.p_prime)


@pytest.mark.parametrize("p", [q for q in TINY_ODD if q < 100])
def test_mont_fma_brute_force_all_triples(p):
    """For every x, y, z the result w lies in [0, P) and w R == x y + z R
    (mod P): REDC of x y (Alg. 2) followed by a modular add of z, which
    Sec. 3.1 notes is the same in Montgomery form.  Checked on w itself,
    not through from_mont, which would hide a missing final reduction."""
    g = np.arange(p, dtype=np.int64)
    xs, ys, zs = (v.ravel() for v in np.meshgrid(g, g, g, indexing="ij"))
    w = oracle.mont_fma(p, xs, ys, zs).astype(np.int64)
    assert np.all((w >= 0) & (w < p))
    assert np.all((w * (R % p) - xs * ys - zs * (R % p)) % p == 0)


@pytest.mark.parametrize("p", TINY_ODD)
def test_to_from_mont_brute_force(p):
    x = np.arange(p, dtype=np.uint32)
    t = oracle.to_mont(p, x).astype(np.int64)
    f = oracle.from_mont(p, x).astype(np.int64)
    assert np.all(t < p) and np.all(f < p)
    assert np.all((t - x.astype(np.int64) * (R % p)) % p == 0)          # x-bar = x R mod P
    assert np.all((f * (R % p) - x.astype(np.int64)) % p == 0)          # f R == x
    assert np.array_equal(oracle.from_mont(p, t), x)


@pytest.mark.parametrize("p", synth.PRIMES)
def test_redc_identity_and_additivity(p):
    """mont_mul(xR, yR) = xyR mod P and (x+y)R = xR + yR (Sec. 3.1)."""
    x = synth.residues(20000, p, 77, 0)
    y = synth.residues(20000, p, 77, 1)
    z = synth.residues(20000, p, 77, 2)
    xm, ym, zm = oracle.to_mont(p, x), oracle.to_mont(p, y), oracle.to_mont(p, z)
    xy = np.array([(int(a) * int(b)) % p for a, b in zip(x, y)], dtype=np.uint32)
    assert np.array_equal(oracle.mont_mul(p, xm, ym), oracle.to_mont(p, xy))
    s = ((x.astype(np.uint64) + y) % p).astype(np.uint32)
    assert np.array_equal(oracle.to_mont(p, s), ((xm.astype(np.uint64) + ym) % p).astype(np.uint32))
    fma = oracle.from_mont(p, oracle.mont_fma(p, xm, ym, zm))
    assert np.array_equal(fma, ((xy.astype(np.uint64) + z) % p).astype(np.uint32))
    c = oracle.setup(p)
    mm = oracle.mont_mul(p, x[:3000], y[:3000])
    for a, b, r in zip(x[:3000].tolist(), y[:3000].tolist(), mm.tolist()):
        assert r == _redc_alg2(a, b, p, c.p_prime)


@pytest.mark.parametrize("p", synth.PRIMES)
def test_adversarial_values(p):
    vals = np.array([0, 1, 2, p - 1, p - 2, R % p, (R * R) % p, p // 2, p // 2 + 1], dtype=np.uint32)
    xs = np.repeat(vals, vals.size)
    ys = np.tile(vals, vals.size)
    c = oracle.setup(p)
    got = oracle.mont_mul(p, xs, ys)
    for a, b, r in zip(xs.tolist(), ys.tolist(), got.tolist()):
        assert r == _redc_alg2(a, b, p, c.p_prime)
    # mont_fma at the same values, with every z: sums past P must wrap
    xs3, zs3 = np.repeat(xs, vals.size), np.tile(vals, xs.size)
    ys3 = np.repeat(ys, vals.size)
    fma = oracle.mont_fma(p, xs3, ys3, zs3)
    for a, b, z, w in zip(xs3.tolist(), ys3.tolist(), zs3.tolist(), fma.tolist()):
        assert w < p and (w * R - a * b - z * R) % p == 0


def test_golden_examples():
    for kind, p, args, expected in _golden_examples():
        if kind == "dft":
            x = [int(v) for v in args[0].split(",")]
            assert oracle.dft(p, x).tolist() == expected
            assert oracle.ntt(p, x).tolist() == expected
            assert oracle.dft(p, expected, inverse=True).tolist() == x
        elif kind == "polymul":
            a = [int(v) for v in args[0].split(",")]
            b = [int(v) for v in args[1].split(",")]
            assert oracle.polymul_schoolbook(p, a, b).tolist() == expected
            assert oracle.polymul_ntt(p, a, b).tolist() == expected
        elif kind == "mont_mul":
            assert oracle.mont_mul(p, [int(args[0])], [int(args[1])]).tolist() == expected
        elif kind == "to_mont":
            assert oracle.to_mont(p, [int(args[0])]).tolist() == expected
        elif kind == "tft":
            k = int(args[0])
            x = [int(v) for v in args[1].split(",")]
            assert oracle.tft(p, x, k).tolist() == expected
            assert oracle.itft(p, expected, k).tolist() == x
        else:
            raise AssertionError(kind)


# ---------------------------------------------------------------- roots of unity

@pytest.mark.parametrize("row", _golden_constants(), ids=lambda r: str(r["p"]))
def test_primitive_root_and_fermat(row):
    p, g = row["p"], row["g"]
    fac = _parse_factors(row["factors"])
    prod = 1
    for q, e in fac.items():
        prod *= q ** e
    assert prod == p - 1
    assert oracle.primitive_root(p) == g
    for q in fac:
        assert pow(g, (p - 1) // q, p) != 1
    for h in range(2, g):                       # every smaller candidate has a smaller order
        assert any(pow(h, (p - 1) // q, p) == 1 for q in fac)
    rnd = random.Random(5)
    for _ in range(200):
        a = rnd.randrange(1, p)
        assert oracle.powmod(a, p - 1, p) == 1       # Fermat
    assert oracle.powmod(g, p - 1, p) == 1


def _small_primes(limit):
    sieve = bytearray([1]) * limit
    sieve[:2] = b"\x00\x00"
    for i in range(2, int(limit ** 0.5) + 1):
        if sieve[i]:
            sieve[i * i::i] = bytearray(len(sieve[i * i::i]))
    return [i for i in range(3, limit) if sieve[i]]


def test_primitive_root_brute_force_small_primes():
    """The smallest primitive root of every odd prime below 5000 is the
    smallest g whose powers g, g^2, ... first return to 1 at exponent P - 1
    (order found by repeated multiplication, no factorisation).  The range
    includes 3631, 4051 and 4733, where P - 1 leaves the square of a prime
    after trial division by the smaller factors and a candidate below the
    true root has order (P - 1) / q: a factoring step that stops one trial
    divisor early accepts it."""
    for p in _small_primes(5000):
        g = 2
        while True:
            x, order = g, 1
            while x != 1:
                x = x * g % p
                order += 1
            if order == p - 1:
                break
            g += 1
        assert oracle.primitive_root(p) == g, p


@pytest.mark.parametrize("p", synth.PRIMES)
def test_roots_of_unity_have_exact_order(p):
    two_adic = ((p - 1) & -(p - 1)).bit_length() - 1
    for k in range(1, two_adic + 1):
        n = 1 << k
        w = oracle.root_of_unity(p, n)
        wi = oracle.root_of_unity(p, n, inverse=True)
        assert pow(w, n, p) == 1 and pow(w, n // 2, p) == p - 1
        assert (w * wi) % p == 1
    with pytest.raises(ValueError):
        oracle.root_of_unity(p, 1 << (two_adic + 1))


# ---------------------------------------------------------------- DFT / NTT

def _horner(coeffs, x, p):
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * x + c) % p
    return acc


@pytest.mark.parametrize("p", TINY_PRIMES + list(synth.PRIMES))
def test_dft_closed_forms(p):
    two_adic = ((p - 1) & -(p - 1)).bit_length() - 1
    for k in range(0, min(two_adic, 6) + 1):
        n = 1 << k
        w = oracle.root_of_unity(p, n)
        delta = np.zeros(n, dtype=np.uint32)
        delta[0] = 1
        assert np.all(oracle.dft(p, delta) == 1)
        ones = np.ones(n, dtype=np.uint32)
        expect = np.zeros(n, dtype=np.uint32)
        expect[0] = n % p
        assert np.array_equal(oracle.dft(p, ones), expect)
        for s in range(n):
            d = np.zeros(n, dtype=np.uint32)
            d[s] = 1
            assert oracle.dft(p, d).tolist() == [pow(w, s * j, p) for j in range(n)]


@pytest.mark.parametrize("p", synth.PRIMES)
@pytest.mark.parametrize("logn", [0, 1, 2, 3, 5, 8, 10])
def test_dft_is_polynomial_evaluation(p, logn):
    n = 1 << logn
    x = synth.residues(n, p, 91, logn)
    w = oracle.root_of_unity(p, n)
    X = oracle.dft(p, x)
    ks = range(n) if n <= 64 else random.Random(logn).sample(range(n), 64)
    xs = x.tolist()
    for k in ks:
        assert X[k] == _horner(xs, pow(w, k, p), p)
    assert np.array_equal(oracle.ntt(p, x), X)
    assert np.array_equal(oracle.dft(p, X, inverse=True), x)
    assert np.array_equal(oracle.ntt(p, X, inverse=True), x)


@pytest.mark.parametrize("p", TINY_PRIMES)
def test_ntt_equals_dft_tiny_primes(p):
    two_adic = ((p - 1) & -(p - 1)).bit_length() - 1
    for k in range(0, min(two_adic, 9) + 1):
        n = 1 << k
        x = synth.residues(n, p, 92, k)
        assert np.array_equal(oracle.ntt(p, x), oracle.dft(p, x))


@pytest.mark.parametrize("p", synth.PRIMES)
def test_convolution_theorem(p):
    n = 256
    a = synth.residues(n, p, 93, 0)
    b = synth.residues(n, p, 93, 1)
    lin = oracle.polymul_schoolbook(p, a, b)
    cyc = np.zeros(n, dtype=np.uint64)
    for k, v in enumerate(lin.tolist()):
        cyc[k % n] = (int(cyc[k % n]) + v) % p
    lhs = oracle.dft(p, cyc.astype(np.uint32))
    rhs = oracle.mulmod_vec(p, oracle.dft(p, a), oracle.dft(p, b))
    assert np.array_equal(lhs, rhs)


# ---------------------------------------------------------------- polynomial products

def _kronecker(a, b, p):
    """Exact product via one big-integer multiplication (Kronecker substitution)."""
    la, lb = len(a), len(b)
    bits = (2 * p.bit_length() + max(la, lb).bit_length() + 1)
    A = sum(int(v) << (bits * i) for i, v in enumerate(a))
    B = sum(int(v) << (bits * i) for i, v in enumerate(b))
    C = A * B
    mask = (1 << bits) - 1
    return [((C >> (bits * k)) & mask) % p for k in range(la + lb - 1)]


@pytest.mark.parametrize("p", synth.PRIMES + (17, 97))
@pytest.mark.parametrize("la,lb", [(1, 1), (1, 7), (2, 3), (5, 5), (31, 17), (64, 64), (100, 3),
                                   (257, 255)])
def test_polymul_against_big_integers(p, la, lb):
    a = synth.residues(la, p, 94, la, lb, 0)
    b = synth.residues(lb, p, 94, la, lb, 1)
    ref = _kronecker(a.tolist(), b.tolist(), p)
    assert oracle.polymul_schoolbook(p, a, b).tolist() == ref
    if (p - 1) % (1 << (la + lb - 2).bit_length()) == 0:
        assert oracle.polymul_ntt(p, a, b).tolist() == ref


@pytest.mark.parametrize("p", synth.PRIMES)
def test_polymul_ntt_equals_schoolbook_sizes(p):
    for la, lb in [(2048, 2048), (1000, 3), (1, 4096), (777, 1234)]:
        a = synth.residues(la, p, 95, la, lb, 0)
        b = synth.residues(lb, p, 95, la, lb, 1)
        assert np.array_equal(oracle.polymul_ntt(p, a, b), oracle.polymul_schoolbook(p, a, b))


def test_polymul_batch_matches_single_products():
    wl = synth.UnevenBatch([synth.P1, synth.P2, synth.P3, synth.P2], [3, 64, 100, 1], [5, 64, 1, 1],
                           (96,))
    for use_ntt in (False, True):
        c = oracle.polymul_batch(wl.primes, wl.a, wl.a_off, wl.la, wl.b, wl.b_off, wl.lb, wl.c_off,
                                 wl.c_size, use_ntt=use_ntt)
        for i in range(len(wl)):
            ao, la = int(wl.a_off[i]), int(wl.la[i])
            bo, lb = int(wl.b_off[i]), int(wl.lb[i])
            co = int(wl.c_off[i])
            ref = _kronecker(wl.a[ao:ao + la].tolist(), wl.b[bo:bo + lb].tolist(), int(wl.primes[i]))
            assert c[co:co + la + lb - 1].tolist() == ref


# ---------------------------------------------------------------- truncated Fourier transform

def _brev(i, bits):
    return int(format(i, "0%db" % bits)[::-1], 2) if bits else 0


@pytest.mark.parametrize("p", synth.PRIMES)
def test_tft_is_the_truncated_dft(p):
    """For every N = 2^K <= 2^10 and every length 1 <= l <= N: the TFT of x
    (l entries) is X_brev(q), q < l, where X_k = sum_{j<l} x_j w^(jk) is
    summed here from the definition (prefix sums over j, in numpy), not by
    any oracle routine."""
    for k in range(0, 11):
        n = 1 << k
        w = int(oracle.root_of_unity(p, n)) if n > 1 else 1
        wpow = np.ones(n, dtype=np.uint64)
        for e in range(1, n):
            wpow[e] = wpow[e - 1] * w % p
        x = synth.residues(n, p, 97, k).astype(np.uint64)
        idx = np.arange(n, dtype=np.uint64)
        order = np.array([_brev(q, k) for q in range(n)])
        X = np.zeros(n, dtype=np.uint64)
        for l in range(1, n + 1):
            j = l - 1
            X = (X + x[j] * wpow[(j * idx) % n]) % p
            got = oracle.tft(p, x[:l].astype(np.uint32), k)
            assert np.array_equal(got, X[order[:l]].astype(np.uint32)), (k, l)


@pytest.mark.parametrize("p", synth.PRIMES)
def test_itft_inverts_tft(p):
    """ITFT(TFT(x)) = x for every l <= N <= 2^10, and TFT(ITFT(y)) = y for
    arbitrary y (the l evaluation points are distinct, so the TFT is a
    bijection on length-l vectors)."""
    for k in range(0, 11):
        n = 1 << k
        for l in range(1, n + 1):
            x = synth.residues(l, p, 98, k, l, 0)
            assert np.array_equal(oracle.itft(p, oracle.tft(p, x, k), k), x), (k, l)
            if l % 7 == 1 or l == n:
                y = synth.residues(l, p, 98, k, l, 1)
                assert np.array_equal(oracle.tft(p, oracle.itft(p, y, k), k), y), (k, l)


@pytest.mark.parametrize("p", synth.PRIMES + (17, 97))
@pytest.mark.parametrize("la,lb", [(1, 1), (1, 2), (2, 2), (3, 2), (5, 5), (9, 8), (31, 17), (33, 32),
                                   (64, 65), (100, 3), (130, 129), (257, 255)])
def test_polymul_tft_against_big_integers(p, la, lb):
    if (p - 1) % (1 << (la + lb - 2).bit_length()) != 0:
        pytest.skip("no root of unity of that order")
    a = synth.residues(la, p, 99, la, lb, 0)
    b = synth.residues(lb, p, 99, la, lb, 1)
    assert oracle.polymul_tft(p, a, b).tolist() == _kronecker(a.tolist(), b.tolist(), p)
