"""GPU parity of the NTT and polynomial-multiplication kernels with the CPU oracle.

Bit-exact: forward and inverse transforms for every supported single-CTA
size and each Fourier prime (natural and bit-reversed order, ragged batch
counts), and products of many shapes, including the 4096 x 2048 batch.
"""
import numpy as np
import pytest

import oracle
from paper_1609_00999_gb300 import synth

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00999_gb300 as m
    from paper_1609_00999_gb300 import build
    build.build()
    return m


def bitrev_perm(logn):
    n = 1 << logn
    return np.array([int(format(k, "0%db" % logn)[::-1], 2) if logn else 0 for k in range(n)], dtype=np.int64)


def oracle_rows(p, x, inverse=False):
    return np.stack([oracle.ntt(p, row, inverse=inverse) for row in x])


@pytest.mark.parametrize("p", synth.PRIMES)
@pytest.mark.parametrize("logn", list(range(0, 15)))
def test_ntt_forward_inverse(m, p, logn):
    n = 1 << logn
    batch = 1 if logn >= 12 else (3 if logn >= 8 else 37)
    x = synth.residues(batch * n, p, 300, logn).reshape(batch, n)
    plan = m.ntt_plan_create(p, logn)
    ref = oracle_rows(p, x)
    d = to_dev(x)
    m.ntt_fwd(plan, d)
    got = to_host(d).reshape(batch, n)
    assert np.array_equal(got, ref)
    m.ntt_inv(plan, d)
    assert np.array_equal(to_host(d).reshape(batch, n), x)
    # bit-reversed order out of the forward / into the inverse
    d = to_dev(x)
    m.ntt_fwd(plan, d, flags=m.NTT_BITREV)
    perm = bitrev_perm(logn)
    assert np.array_equal(to_host(d).reshape(batch, n), ref[:, perm])
    m.ntt_inv(plan, d, flags=m.NTT_BITREV)
    assert np.array_equal(to_host(d).reshape(batch, n), x)
    # inverse alone against the oracle's inverse
    d = to_dev(x)
    m.ntt_inv(plan, d)
    assert np.array_equal(to_host(d).reshape(batch, n), oracle_rows(p, x, inverse=True))


@pytest.mark.parametrize("logn", [11, 12, 13, 14])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_ntt_natural_order_rows_aligned_and_not(m, logn, offset):
    """Natural-order transforms of several rows whose data start 16-byte
    aligned (rows move as uint4, bank-conflict-free bit-reversed positions)
    or 4 / 12 bytes past it (one word at a time)."""
    import torch
    p = synth.P3
    n, batch = 1 << logn, 3
    x = synth.residues(batch * n, p, 302, logn, offset).reshape(batch, n)
    plan = m.ntt_plan_create(p, logn)
    buf = torch.zeros(batch * n + 4, dtype=torch.int32, device="cuda")
    d = buf[offset:offset + batch * n]
    d.copy_(to_dev(x.ravel()))
    m.ntt_fwd(plan, d)
    assert np.array_equal(to_host(d).reshape(batch, n), oracle_rows(p, x))
    m.ntt_inv(plan, d)
    assert np.array_equal(to_host(d).reshape(batch, n), x)
    assert not to_host(buf[:offset]).any() and not to_host(buf[offset + batch * n:]).any()


@pytest.mark.parametrize("p", synth.PRIMES)
@pytest.mark.parametrize("la,lb", [(1, 1), (1, 2), (2, 1), (3, 5), (16, 16), (17, 9), (100, 29), (255, 257),
                                   (1024, 1024), (1, 4096), (2048, 2048), (3000, 1000), (5000, 3193),
                                   (8192, 8192), (1, 16384), (12000, 4385)])
def test_polymul_single(m, p, la, lb):
    a = synth.residues(la, p, 301, la, lb, 0)
    b = synth.residues(lb, p, 301, la, lb, 1)
    got = to_host(m.polymul(p, to_dev(a), to_dev(b)))
    ref = oracle.polymul_schoolbook(p, a, b) if la * lb <= (1 << 22) else oracle.polymul_ntt(p, a, b)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("p", synth.PRIMES)
@pytest.mark.parametrize("count,la,lb", [(1, 7, 7), (5, 64, 64), (33, 100, 28), (257, 31, 33), (19, 700, 300),
                                         (3, 4000, 4000)])
def test_polymul_many_shapes(m, p, count, la, lb):
    a = synth.residues(count * la, p, 302, count, la, lb, 0).reshape(count, la)
    b = synth.residues(count * lb, p, 302, count, la, lb, 1).reshape(count, lb)
    got = to_host(m.polymul_many(p, to_dev(a), to_dev(b))).reshape(count, la + lb - 1)
    for i in range(count):
        assert np.array_equal(got[i], oracle.polymul_schoolbook(p, a[i], b[i])), i


def test_polymul_batch_4096x2048(m):
    """4096 products of length-2048 polynomials mod P1 (N = 4096), every output checked."""
    p, a, b = synth.batch_uniform()
    count, L = a.shape
    got = to_host(m.polymul_many(p, to_dev(a), to_dev(b))).reshape(count, 2 * L - 1)
    off = np.arange(count, dtype=np.uint64) * L
    lens = np.full(count, L, dtype=np.uint64)
    c_off = np.arange(count, dtype=np.uint64) * (2 * L - 1)
    ref = oracle.polymul_batch(np.full(count, p, dtype=np.uint32), a.ravel(), off, lens, b.ravel(), off, lens,
                               c_off, count * (2 * L - 1), use_ntt=True).reshape(count, 2 * L - 1)
    assert np.array_equal(got, ref)
    for i in (0, 1, 2047, 4095):
        assert np.array_equal(got[i], oracle.polymul_schoolbook(p, a[i], b[i]))


def test_polymul_adversarial_values(m):
    for p in synth.PRIMES:
        for v in (0, 1, p - 1, p // 2):
            a = np.full(1500, v, dtype=np.uint32)
            b = np.full(1700, p - 1, dtype=np.uint32)
            got = to_host(m.polymul(p, to_dev(a), to_dev(b)))
            assert np.array_equal(got, oracle.polymul_schoolbook(p, a, b))


@pytest.mark.parametrize("logn", [1, 2, 5, 11, 12, 14])
def test_ntt_extreme_inputs(m, logn):
    """Inputs at the top of the residue range: the forward passes keep values
    in [0, 2P), so P - 1 everywhere (and alternating with 0) drives the
    intermediate sums closest to 2^32 for the largest prime."""
    n = 1 << logn
    for p in synth.PRIMES:
        x = np.stack([np.full(n, p - 1, dtype=np.uint32),
                      np.where(np.arange(n) % 2 == 0, p - 1, 0).astype(np.uint32),
                      np.where(np.arange(n) < n // 2, p - 1, p - 2).astype(np.uint32)])
        plan = m.ntt_plan_create(p, logn)
        d = to_dev(x)
        m.ntt_fwd(plan, d)
        assert np.array_equal(to_host(d).reshape(3, n), oracle_rows(p, x))
        m.ntt_inv(plan, d)
        assert np.array_equal(to_host(d).reshape(3, n), x)


def test_polymul_errors(m):
    import torch
    d = to_dev(np.zeros(8, dtype=np.uint32))
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    with pytest.raises(m.MontError) as ex:
        m.polymul(synth.P1, e, d, out=to_dev(np.zeros(7, dtype=np.uint32)))
    assert ex.value.code == m.MONT_EINVAL
    with pytest.raises(m.MontError) as ex:
        m.ntt_plan_create(synth.P3, 25)           # 2^25 does not divide P3 - 1
    assert ex.value.code == m.MONT_ERANGE
    with pytest.raises(m.MontError) as ex:
        m.ntt_plan_create(synth.P1 + 2, 4)        # not prime
    assert ex.value.code == m.MONT_EINVAL
    big = to_dev(np.zeros(12, dtype=np.uint32))
    # output overlapping an input is rejected before any launch
    rc = m.lib().polymul(synth.P1, big.data_ptr(), 4, big.data_ptr() + 16, 4, big.data_ptr() + 8, None)
    assert rc == m.MONT_EINVAL
