"""GPU parity of the elementwise Montgomery kernels against the CPU oracle.

Bit-exact (integer work): to_mont, from_mont, mont_mul, mont_fma through the C
ABI, at sizes spanning many tiles with ragged tails, on misaligned and
in-place operands, on adversarial residues, and at the full 2^28-element
workload for each of the three Fourier primes.
"""
import numpy as np
import pytest

import oracle
from paper_1609_00999_gb300 import synth

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 3, 4, 5, 7, 8, 31, 33, 255, 256, 257, 1023, 4097, 65535, 65536, 65537,
         256 * 2 * 1216 * 4 + 13, 1 << 20, (1 << 22) + 3]


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00999_gb300 as m
    from paper_1609_00999_gb300 import build
    build.build()
    return m


def test_small_config_roundtrip(m):
    """65,536 pairs mod P1: to_mont a, b -> mont_mul -> from_mont == (a b) mod P."""
    p, a, b = synth.elementwise_small()
    ctx = m.mont_setup(p)
    da, db = to_dev(a), to_dev(b)
    am, bm = m.to_mont(ctx, da), m.to_mont(ctx, db)
    prod = m.from_mont(ctx, m.mont_mul(ctx, am, bm))
    assert np.array_equal(to_host(am), oracle.to_mont(p, a))
    assert np.array_equal(to_host(bm), oracle.to_mont(p, b))
    assert np.array_equal(to_host(prod), oracle.mulmod_vec(p, a, b))


@pytest.mark.parametrize("p", synth.PRIMES)
@pytest.mark.parametrize("n", SIZES)
def test_ops_match_oracle(m, p, n):
    a = synth.residues(n, p, 200, n, 0)
    b = synth.residues(n, p, 200, n, 1)
    c = synth.residues(n, p, 200, n, 2)
    ctx = m.mont_setup(p)
    da, db, dc = to_dev(a), to_dev(b), to_dev(c)
    assert np.array_equal(to_host(m.to_mont(ctx, da)), oracle.to_mont(p, a))
    assert np.array_equal(to_host(m.from_mont(ctx, da)), oracle.from_mont(p, a))
    assert np.array_equal(to_host(m.mont_mul(ctx, da, db)), oracle.mont_mul(p, a, b))
    assert np.array_equal(to_host(m.mont_fma(ctx, da, db, dc)), oracle.mont_fma(p, a, b, c))


@pytest.mark.parametrize("p", synth.PRIMES)
def test_adversarial_residues(m, p):
    vals = np.array([0, 1, 2, 3, p - 1, p - 2, p - 3, (1 << 32) % p, ((1 << 32) % p) ** 2 % p,
                     p // 2, p // 2 + 1, (p + 1) // 3], dtype=np.uint32)
    a = np.repeat(vals, vals.size)
    b = np.tile(vals, vals.size)
    c = np.roll(a, 5)
    ctx = m.mont_setup(p)
    da, db, dc = to_dev(a), to_dev(b), to_dev(c)
    assert np.array_equal(to_host(m.mont_mul(ctx, da, db)), oracle.mont_mul(p, a, b))
    assert np.array_equal(to_host(m.mont_fma(ctx, da, db, dc)), oracle.mont_fma(p, a, b, c))
    assert np.array_equal(to_host(m.to_mont(ctx, da)), oracle.to_mont(p, a))
    assert np.array_equal(to_host(m.from_mont(ctx, da)), oracle.from_mont(p, a))


@pytest.mark.parametrize("offs", [(1, 0, 0, 0), (0, 1, 2, 3), (3, 3, 3, 3), (2, 0, 1, 2)])
def test_misaligned_operands(m, offs):
    """Sub-views that are not 16-byte aligned take the scalar path; results are unchanged."""
    p, n = synth.P2, 100003
    a = synth.residues(n + 4, p, 201, 0)
    b = synth.residues(n + 4, p, 201, 1)
    c = synth.residues(n + 4, p, 201, 2)
    ctx = m.mont_setup(p)
    da, db, dc = to_dev(a), to_dev(b), to_dev(c)
    out = to_dev(np.zeros(n + 4, dtype=np.uint32))
    oa, ob, oc, oo = offs
    m.mont_fma(ctx, da[oa:oa + n], db[ob:ob + n], dc[oc:oc + n], out=out[oo:oo + n])
    assert np.array_equal(to_host(out)[oo:oo + n], oracle.mont_fma(p, a[oa:oa + n], b[ob:ob + n], c[oc:oc + n]))
    m.mont_mul(ctx, da[oa:oa + n], db[ob:ob + n], out=out[oo:oo + n])
    assert np.array_equal(to_host(out)[oo:oo + n], oracle.mont_mul(p, a[oa:oa + n], b[ob:ob + n]))


def test_in_place(m):
    p, n = synth.P3, 300007
    a = synth.residues(n, p, 202, 0)
    b = synth.residues(n, p, 202, 1)
    ctx = m.mont_setup(p)
    da, db = to_dev(a), to_dev(b)
    m.mont_mul(ctx, da, db, out=da)
    assert np.array_equal(to_host(da), oracle.mont_mul(p, a, b))
    m.to_mont(ctx, db, out=db)
    assert np.array_equal(to_host(db), oracle.to_mont(p, b))


def test_partial_overlap_rejected(m):
    ctx = m.mont_setup(synth.P1)
    d = to_dev(np.zeros(1024, dtype=np.uint32))
    with pytest.raises(m.MontError) as e:
        m.mont_mul(ctx, d[0:512], d[0:512], out=d[1:513])
    assert e.value.code == m.MONT_EINVAL


def test_explicit_stream(m):
    import torch
    p, n = synth.P1, 1 << 18
    a = synth.residues(n, p, 203, 0)
    b = synth.residues(n, p, 203, 1)
    ctx = m.mont_setup(p)
    s = torch.cuda.Stream()
    da, db = to_dev(a), to_dev(b)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        out = m.mont_mul(ctx, da, db, stream=s)
    s.synchronize()
    assert np.array_equal(to_host(out), oracle.mont_mul(p, a, b))


@pytest.mark.parametrize("prime_index", [0, 1, 2])
def test_full_size_elementwise(m, prime_index):
    """The 2^28-element HBM-bound workload, every output compared with the oracle."""
    import torch
    p, (a, b, c) = synth.elementwise_large(prime_index)
    ctx = m.mont_setup(p)
    da, db, dc = to_dev(a), to_dev(b), to_dev(c)
    out = torch.empty_like(da)
    m.mont_mul(ctx, da, db, out=out)
    assert np.array_equal(to_host(out), oracle.mont_mul(p, a, b))
    m.mont_fma(ctx, da, db, dc, out=out)
    assert np.array_equal(to_host(out), oracle.mont_fma(p, a, b, c))
    del da, db, dc, out
    torch.cuda.empty_cache()


def test_pinned_host_operands_zero_copy(m):
    """Kernels on pinned host buffers (read/written in place over the CPU-GPU
    link) give the same results as on device buffers."""
    import torch
    p, n = synth.P1, (1 << 20) + 5
    a = synth.residues(n, p, 204, 0)
    b = synth.residues(n, p, 204, 1)
    c = synth.residues(n, p, 204, 2)
    ctx = m.mont_setup(p)
    ha, hb, hc = (torch.from_numpy(x.view(np.int32)).pin_memory() for x in (a, b, c))
    ho = torch.empty(n, dtype=torch.int32).pin_memory()
    m.mont_mul(ctx, ha, hb, out=ho)
    torch.cuda.synchronize()
    assert np.array_equal(ho.numpy().view(np.uint32), oracle.mont_mul(p, a, b))
    m.mont_fma(ctx, ha, hb, hc, out=ho)
    torch.cuda.synchronize()
    assert np.array_equal(ho.numpy().view(np.uint32), oracle.mont_fma(p, a, b, c))
    dout = torch.empty(n, dtype=torch.int32, device="cuda")
    m.mont_mul(ctx, ha, to_dev(b), out=dout)                   # host and device operands mixed
    assert np.array_equal(to_host(dout), oracle.mont_mul(p, a, b))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 31, 1023, 4097, 65537, (1 << 22) + 3])
@pytest.mark.parametrize("p", synth.PRIMES)
def test_check_residues(m, p, n):
    """mont_check_residues agrees with the definition (every word < p) on
    aligned and misaligned buffers, with one planted non-residue at the head,
    the middle or the ragged tail, and with the largest residue p - 1."""
    import torch
    x = synth.residues(n + 1, p, 210, n)
    d = to_dev(x)
    for view in (d[:n], d[1:n + 1]):                           # 16-byte aligned, then 4 bytes off
        assert m.check_residues(p, view)
        for pos in sorted({0, n // 2, n - 1}):
            for bad in (p, 0xFFFFFFFF):
                host = view.cpu().numpy().view(np.uint32).copy()
                host[pos] = bad
                v2 = view.clone() if view.data_ptr() % 16 == 0 else d.clone()[1:n + 1]
                v2.copy_(torch.from_numpy(host.view(np.int32)))
                assert not (host < p).all()
                assert not m.check_residues(p, v2), (pos, bad)
    top = torch.full((n,), p - 1, dtype=torch.int32, device="cuda")
    assert m.check_residues(p, top)
    assert m.check_residues(p, torch.empty(0, dtype=torch.int32, device="cuda"))


def test_check_residues_pinned_and_errors(m):
    import torch
    p = synth.P2
    x = synth.residues(70001, p, 211, 0)
    h = torch.from_numpy(x.view(np.int32)).pin_memory()
    assert m.check_residues(p, h)
    h[70000] = p
    assert not m.check_residues(p, h)
    with pytest.raises(m.MontError) as e:
        m.check_residues(4, h)
    assert e.value.code == m.MONT_EINVAL
