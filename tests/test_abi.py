"""CPU-side checks of the C ABI: the library builds, loads and exports every
declared symbol, host-side set-up agrees with the oracle, and argument errors
are rejected on the host before any device work (no GPU needed)."""
import ctypes

import pytest

import oracle
from paper_1609_00999_gb300 import build as gbuild
from paper_1609_00999_gb300 import synth

from helpers import header_functions


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    import paper_1609_00999_gb300 as m
    return m.lib()


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert "mont_setup" in names and "mont_mul" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("p", list(synth.PRIMES) + [3, 5, 17, 97, 65537, 2 ** 31 - 1])
def test_mont_setup_matches_oracle(L, p):
    import paper_1609_00999_gb300 as m
    ctx = m.mont_setup(p)
    ref = oracle.setup(p)
    assert (ctx.p, ctx.p_prime, ctx.r_mod_p, ctx.r2_mod_p) == (ref.p, ref.p_prime, ref.r_mod_p, ref.r2_mod_p)


@pytest.mark.parametrize("p", [0, 1, 2, 4, 2 ** 31, 2 ** 31 + 1, 3 * 2 ** 30 + 1, 2 ** 32 - 1])
def test_mont_setup_rejects(L, p):
    import paper_1609_00999_gb300 as m
    with pytest.raises(m.MontError) as e:
        m.mont_setup(p)
    assert e.value.code == m.MONT_EINVAL


def test_host_side_argument_errors(L):
    import paper_1609_00999_gb300 as m
    ctx = m.mont_setup(synth.P1)
    bad = m.MontCtx(ctx.p, ctx.p_prime ^ 1, ctx.r_mod_p, ctx.r2_mod_p)
    buf = ctypes.c_void_p(0x100000)
    assert L.mont_mul(None, buf, buf, buf, 4, None) == m.MONT_EINVAL
    assert L.mont_mul(ctypes.byref(bad), buf, buf, buf, 4, None) == m.MONT_EINVAL
    assert L.mont_mul(ctypes.byref(ctx), None, buf, buf, 4, None) == m.MONT_EINVAL
    # partial overlap of output with an input
    assert L.mont_mul(ctypes.byref(ctx), ctypes.c_void_p(0x100000), buf, ctypes.c_void_p(0x100004), 4,
                      None) == m.MONT_EINVAL
    # n == 0 is a no-op
    assert L.mont_mul(ctypes.byref(ctx), None, None, None, 0, None) == m.MONT_OK
    assert L.mont_fma(ctypes.byref(ctx), buf, buf, None, buf, 4, None) == m.MONT_EINVAL
    assert L.to_mont(None, buf, buf, 4, None) == m.MONT_EINVAL
    # the residue check: bad moduli and a NULL buffer fail before any device work
    for p in (0, 1, 2, 4, 2 ** 31, 2 ** 32 - 1):
        assert L.mont_check_residues(p, buf, 4, None) == m.MONT_EINVAL
    assert L.mont_check_residues(synth.P1, None, 4, None) == m.MONT_EINVAL
    assert L.mont_check_residues(synth.P1, None, 0, None) == m.MONT_OK
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(m.strerror(code), str)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    import paper_1609_00999_gb300._binding as b
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(b, "_lib", None)
    with pytest.raises(RuntimeError):
        b.lib()


def test_one_shot_batch_host_checks(L):
    """polymul_batch sizes its workspace and rejects bad arguments on the
    host, before any device work (descriptor addresses are not touched)."""
    import paper_1609_00999_gb300 as m
    a0, c0 = 0x100000, 0x40000000

    def desc(la, lb, k):
        return m.PolymulDesc(a0 + k * 0x1000000, a0 + k * 0x1000000 + 0x800000, c0 + k * 0x1000000, la, lb,
                             synth.P1, 0)

    descs = [desc(100, 50, 0), desc(20000, 20000, 1), desc(3, 1, 2)]
    need = m.polymul_batch_workspace_bytes(descs)
    assert need >= 2 * (1 << 16) * 4                     # the N = 2^16 product's scratch
    assert m.polymul_batch_workspace_bytes(descs[:1]) < need
    assert m.polymul_batch_workspace_bytes([]) == 0
    assert m.polymul_batch_workspace_bytes([desc(0, 5, 0)]) == 0
    arr = (m.PolymulDesc * 3)(*descs)
    ws = ctypes.c_void_p(0x7f0000000000)
    assert L.polymul_batch(arr, 3, None, need, None) == m.MONT_EINVAL
    assert L.polymul_batch(arr, 3, ws, need - 1, None) == m.MONT_EINVAL
    assert L.polymul_batch(arr, 3, ctypes.c_void_p(0x7f0000000010), need, None) == m.MONT_EINVAL
    assert L.polymul_batch(None, 3, ws, need, None) == m.MONT_EINVAL
    assert L.polymul_batch(None, 0, None, 0, None) == m.MONT_OK
    bad = (m.PolymulDesc * 1)(desc(5, 0, 0))
    assert L.polymul_batch(bad, 1, ws, need, None) == m.MONT_EINVAL
    assert L.polymul_batch_check(None, None) == m.MONT_EINVAL


def test_int_probe_argument_errors(L):
    """The integer-pipe probe rejects bad arguments on the host, before any launch."""
    import paper_1609_00999_gb300 as m
    sink = ctypes.c_void_p(0x100000)
    ops = ctypes.c_uint64(0)
    assert L.mont_int_probe(99, synth.P1, 4, 1, sink, ctypes.byref(ops), None) == m.MONT_EINVAL   # unknown kind
    assert L.mont_int_probe(-1, synth.P1, 4, 1, sink, ctypes.byref(ops), None) == m.MONT_EINVAL
    assert L.mont_int_probe(4, synth.P1, 4, 1, None, ctypes.byref(ops), None) == m.MONT_EINVAL     # no sink
    assert L.mont_int_probe(4, synth.P1, 0, 1, sink, ctypes.byref(ops), None) == m.MONT_EINVAL     # no work
    for p in (0, 2, 2 ** 31 + 1):
        assert L.mont_int_probe(4, p, 4, 1, sink, ctypes.byref(ops), None) == m.MONT_EINVAL
    assert sorted(m.PROBE_KINDS.values()) == list(range(10))
