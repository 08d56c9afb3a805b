"""GPU parity of the large-N path (N = 2^15 .. 2^24: column / row / column
kernels through HBM scratch) with the CPU oracle, bit-exact."""
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
    k = np.arange(1 << logn, dtype=np.int64)
    r = np.zeros_like(k)
    for b in range(logn):
        r |= ((k >> b) & 1) << (logn - 1 - b)
    return r


CASES = [(synth.P1, k) for k in range(15, 23)] + [(synth.P2, 15), (synth.P2, 19), (synth.P3, 17), (synth.P3, 21),
                                                 (synth.P3, 24)]


@pytest.mark.parametrize("p,logn", CASES)
def test_large_ntt(m, p, logn):
    n = 1 << logn
    batch = 2 if logn <= 17 else 1
    x = synth.residues(batch * n, p, 400, logn).reshape(batch, n)
    ref = np.stack([oracle.ntt(p, row) for row in x])
    plan = m.ntt_plan_create(p, logn)
    d = to_dev(x)
    m.ntt_fwd(plan, d)
    assert np.array_equal(to_host(d).reshape(batch, n), ref)
    m.ntt_inv(plan, d)
    assert np.array_equal(to_host(d).reshape(batch, n), x)
    d = to_dev(x)
    m.ntt_fwd(plan, d, flags=m.NTT_BITREV)
    assert np.array_equal(to_host(d).reshape(batch, n), ref[:, bitrev_perm(logn)])
    m.ntt_inv(plan, d, flags=m.NTT_BITREV)
    assert np.array_equal(to_host(d).reshape(batch, n), x)


@pytest.mark.parametrize("p,la,lb", [(synth.P1, 8193, 8192), (synth.P1, 16384, 16385), (synth.P2, 30000, 20000),
                                     (synth.P3, 65536, 65536), (synth.P1, 100000, 31073), (synth.P2, 1, 40000),
                                     (synth.P1, 1 << 20, 1 << 20), (synth.P3, 700000, 123457),
                                     (synth.P2, 300000, 100001)])
def test_large_polymul(m, p, la, lb):
    a = synth.residues(la, p, 401, la, lb, 0)
    b = synth.residues(lb, p, 401, la, lb, 1)
    got = to_host(m.polymul(p, to_dev(a), to_dev(b)))
    ref = oracle.polymul_ntt(p, a, b)
    assert np.array_equal(got, ref)
    if la * lb <= (1 << 27):
        idx = [0, 1, la // 2, la + lb - 2]
        sb = oracle.polymul_schoolbook(p, a, b)
        assert np.array_equal(got[idx], sb[idx])


@pytest.mark.parametrize("p", synth.PRIMES)
def test_large_extreme_inputs(m, p):
    """P - 1 everywhere through the column / row kernels (forward values are
    lazy between them)."""
    la, lb = 20000, 13000
    a = np.full(la, p - 1, dtype=np.uint32)
    b = np.full(lb, p - 1, dtype=np.uint32)
    got = to_host(m.polymul(p, to_dev(a), to_dev(b)))
    assert np.array_equal(got, oracle.polymul_ntt(p, a, b))
    for logn in (16, 20):                         # register and shared-memory column passes
        x = np.full((1, 1 << logn), p - 1, dtype=np.uint32)
        plan = m.ntt_plan_create(p, logn)
        d = to_dev(x)
        m.ntt_fwd(plan, d)
        assert np.array_equal(to_host(d).reshape(1, -1), np.stack([oracle.ntt(p, x[0])]))
        m.ntt_inv(plan, d)
        assert np.array_equal(to_host(d).reshape(1, -1), x)


def test_large_polymul_many_and_chunked_workspace(m):
    import torch
    p, count, la, lb = synth.P2, 5, 20000, 12001
    a = synth.residues(count * la, p, 402, 0).reshape(count, la)
    b = synth.residues(count * lb, p, 402, 1).reshape(count, lb)
    ref = np.stack([oracle.polymul_ntt(p, a[i], b[i]) for i in range(count)])
    got = to_host(m.polymul_many(p, to_dev(a), to_dev(b))).reshape(count, la + lb - 1)
    assert np.array_equal(got, ref)
    per = m.polymul_workspace_bytes(la, lb, 1)
    assert per == 2 * 32768 * 4 and m.polymul_workspace_bytes(la, lb, count) == count * per
    ws = torch.empty(2 * per // 4 + 7, dtype=torch.int32, device="cuda")   # room for two products: 3 chunks
    got = to_host(m.polymul_many_ws(p, to_dev(a), to_dev(b), ws)).reshape(count, la + lb - 1)
    assert np.array_equal(got, ref)
    small = torch.empty(per // 4 - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(m.MontError) as e:
        m.polymul_many_ws(p, to_dev(a), to_dev(b), small)
    assert e.value.code == m.MONT_EINVAL


# Single-call products of N = 2^15 .. 2^18 on both sides of the row counts
# of the truncated transforms (rows of 2^12 up to N = 2^16, 2^13 for 2^17,
# 2^14 for 2^18; a product computes ceil(lc / row) rows when that is fewer
# than all of them): the first and last row counts that save a row, exact
# multiples of the row, one past, and asymmetric operands.
TFT_SINGLE = [(16385, 1), (20000, 5000), (14336, 14337), (14337, 14337), (30000, 2769), (1, 32769),
              (40000, 1), (32768, 28673), (65536, 1), (70000, 1), (61440, 61441), (100000, 31073),
              (140000, 1), (180000, 20001), (200000, 50000)]


@pytest.mark.parametrize("la,lb", TFT_SINGLE)
def test_truncated_single_products(m, la, lb):
    p = synth.PRIMES[(la + lb) % 3]
    a = synth.residues(la, p, 320, la, lb, 0)
    b = synth.residues(lb, p, 320, la, lb, 1)
    ref = oracle.polymul_ntt(p, a, b)
    assert np.array_equal(to_host(m.polymul(p, to_dev(a), to_dev(b))), ref)
    if la + lb <= 120000:                       # three at once, each against the oracle
        import torch
        a3 = np.stack([a, np.roll(a, 1), np.roll(a, 2)])
        b3 = np.stack([b, np.roll(b, 3), np.roll(b, 5)])
        got = to_host(m.polymul_many(p, to_dev(a3), to_dev(b3))).reshape(3, la + lb - 1)
        for i in range(3):
            assert np.array_equal(got[i], oracle.polymul_ntt(p, a3[i], b3[i])), i


@pytest.mark.parametrize("p,logn,rows", [(synth.P1, 19, 3), (synth.P2, 20, 2), (synth.P3, 21, 2)])
def test_large_ntt_several_rows(m, p, logn, rows):
    """Several rows of the direct column tiles and row kernels in one call
    (the product index of the grid), each row against the oracle."""
    n = 1 << logn
    x = synth.residues(rows * n, p, 410, logn, rows).reshape(rows, n)
    plan = m.ntt_plan_create(p, logn)
    d = to_dev(x)
    m.ntt_fwd(plan, d)
    got = to_host(d).reshape(rows, n)
    for i in range(rows):
        assert np.array_equal(got[i], oracle.ntt(p, x[i])), i
    m.ntt_inv(plan, d)
    assert np.array_equal(to_host(d).reshape(rows, n), x)


@pytest.mark.parametrize("p,la,lb", [(synth.P2, 200000, 100000), (synth.P1, 400000, 300000)])
def test_large_polymul_many_split_sizes(m, p, la, lb):
    """Two products of N = 2^19 and 2^20 (rows of 2^12) in one call, each
    against the oracle."""
    count = 2
    a = synth.residues(count * la, p, 411, la, lb, 0).reshape(count, la)
    b = synth.residues(count * lb, p, 411, la, lb, 1).reshape(count, lb)
    got = to_host(m.polymul_many(p, to_dev(a), to_dev(b))).reshape(count, la + lb - 1)
    for i in range(count):
        assert np.array_equal(got[i], oracle.polymul_ntt(p, a[i], b[i])), i
