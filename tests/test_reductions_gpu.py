"""GPU parity of the other two reductions of Sec. 3.1 with the oracle:
Barrett (Alg. 1) against (a b) mod P, and Montgomery over Fourier primes
(Alg. 3) against a b R^-1 mod P, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1609_00999_gb300 import synth

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

FOURIER_OK = [synth.P2, synth.P3, 998244353, 167772161, 469762049]   # c 2^n + 1, 2n >= 32, P < 2^30


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00999_gb300 as m
    from paper_1609_00999_gb300 import build
    build.build()
    return m


def adversarial(p):
    return np.array([0, 1, 2, p - 1, p - 2, p // 2, (1 << 32) % p, p // 3], dtype=np.uint32)


@pytest.mark.parametrize("p", list(synth.PRIMES) + [3, 17, 97, 65537, 2 ** 31 - 1, 1000000007])
@pytest.mark.parametrize("n", [1, 7, 4096 + 3, (1 << 20) + 1])
def test_barrett_matches_mulmod(m, p, n):
    a = synth.residues(n, p, 800, n, 0)
    b = synth.residues(n, p, 800, n, 1)
    got = to_host(m.barrett_mulmod(p, to_dev(a), to_dev(b)))
    assert np.array_equal(got, oracle.mulmod_vec(p, a, b))
    v = adversarial(p)
    x, y = np.repeat(v, v.size), np.tile(v, v.size)
    assert np.array_equal(to_host(m.barrett_mulmod(p, to_dev(x), to_dev(y))), oracle.mulmod_vec(p, x, y))


@pytest.mark.parametrize("p", FOURIER_OK)
@pytest.mark.parametrize("n", [1, 5, (1 << 20) + 3])
def test_fourier_redc_matches_redc(m, p, n):
    a = synth.residues(n, p, 801, n, 0)
    b = synth.residues(n, p, 801, n, 1)
    ctx = m.mont_setup(p)
    got = to_host(m.fourier_redc_mul(ctx, to_dev(a), to_dev(b)))
    assert np.array_equal(got, oracle.mont_mul(p, a, b))
    v = adversarial(p)
    x, y = np.repeat(v, v.size), np.tile(v, v.size)
    assert np.array_equal(to_host(m.fourier_redc_mul(ctx, to_dev(x), to_dev(y))), oracle.mont_mul(p, x, y))


@pytest.mark.parametrize("p", [synth.P1, 1000000007, 2 ** 31 - 1])
def test_fourier_redc_rejects_out_of_range_primes(m, p):
    ctx = m.mont_setup(p)
    d = to_dev(np.ones(8, dtype=np.uint32))
    with pytest.raises(m.MontError) as e:
        m.fourier_redc_mul(ctx, d, d)
    assert e.value.code == m.MONT_ERANGE


@pytest.mark.parametrize("p", [synth.P2, synth.P3, 998244353])
@pytest.mark.parametrize("count,la,lb", [(1, 1, 1), (37, 100, 29), (5, 1000, 1024), (4, 2048, 2048),
                                         (2, 5000, 3193), (1, 8192, 8192)])
def test_polymul_fourier_twiddles_match_oracle(m, p, count, la, lb):
    """Fused products with the Alg. 3 twiddle / scaling / pointwise multiply:
    bit-exact against the oracle and equal to the Alg. 2 kernels' output."""
    a = synth.residues(count * la, p, 802, count, la, lb, 0).reshape(count, la)
    b = synth.residues(count * lb, p, 802, count, la, lb, 1).reshape(count, lb)
    da, db = to_dev(a), to_dev(b)
    got = to_host(m.polymul_many_fourier(p, da, db)).reshape(count, la + lb - 1)
    assert np.array_equal(got, to_host(m.polymul_many(p, da, db)).reshape(count, la + lb - 1))
    for i in sorted({0, count - 1}):
        ref = oracle.polymul_schoolbook(p, a[i], b[i]) if la * lb <= (1 << 22) else oracle.polymul_ntt(p, a[i], b[i])
        assert np.array_equal(got[i], ref)


@pytest.mark.parametrize("p", [synth.P2, synth.P3])
def test_polymul_fourier_extreme_inputs(m, p):
    a = np.full((2, 3000), p - 1, dtype=np.uint32)
    b = np.full((2, 2000), p - 1, dtype=np.uint32)
    b[1, ::2] = 0
    got = to_host(m.polymul_many_fourier(p, to_dev(a), to_dev(b))).reshape(2, 4999)
    for i in range(2):
        assert np.array_equal(got[i], oracle.polymul_schoolbook(p, a[i], b[i]))


def test_polymul_fourier_rejects(m):
    d = to_dev(np.ones((1, 64), dtype=np.uint32))
    for p in (synth.P1, 12289):                 # P >= 2^30; 12289 = 3 2^12 + 1 has 2n < 32
        with pytest.raises(m.MontError) as e:
            m.polymul_many_fourier(p, d, d)
        assert e.value.code == m.MONT_ERANGE
    big = to_dev(np.ones((1, 9000), dtype=np.uint32))  # N = 2^15: beyond the single-CTA kernels
    with pytest.raises(m.MontError) as e:
        m.polymul_many_fourier(synth.P2, big, big)
    assert e.value.code == m.MONT_EUNSUPPORTED
