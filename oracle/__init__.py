"""CPU oracle for the Montgomery / NTT / polymul path (ctypes over ``liboracle.so``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg (``bench.py``) may import this package.  It
shares no code with the CUDA library in ``paper_1609_00999_gb300``; neither
imports the other.

Every result is computed from its definition with 64-bit ``%`` (see
``oracle.h``): mulmod, the Montgomery residue map i -> iR mod P and what REDC
returns, x y R^-1 mod P (Meng, Sec. 3.1, Alg. 2), the direct DFT over Z_P
and schoolbook convolution.  R = 2^32.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


class OrCtx(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint32), ("p_prime", ctypes.c_uint32), ("r_inv", ctypes.c_uint32),
                ("r_mod_p", ctypes.c_uint32), ("r2_mod_p", ctypes.c_uint32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB: load another build of oracle.c instead (the mutation
        # test loads copies with planted mistakes to show the pins catch them).
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        L.or_setup.argtypes = [ctypes.c_uint32, ctypes.POINTER(OrCtx)]
        L.or_setup.restype = ctypes.c_int
        for name in ("or_mulmod",):
            getattr(L, name).argtypes = [ctypes.c_uint32] * 3
            getattr(L, name).restype = ctypes.c_uint32
        L.or_powmod.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
        L.or_powmod.restype = ctypes.c_uint32
        L.or_invmod.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_invmod.restype = ctypes.c_uint64
        for name in ("or_to_mont", "or_from_mont"):
            getattr(L, name).argtypes = [ctypes.POINTER(OrCtx), ctypes.c_uint32]
            getattr(L, name).restype = ctypes.c_uint32
        L.or_mont_mul.argtypes = [ctypes.POINTER(OrCtx), ctypes.c_uint32, ctypes.c_uint32]
        L.or_mont_mul.restype = ctypes.c_uint32
        L.or_mont_fma.argtypes = [ctypes.POINTER(OrCtx)] + [ctypes.c_uint32] * 3
        L.or_mont_fma.restype = ctypes.c_uint32
        for name in ("or_to_mont_vec", "or_from_mont_vec"):
            getattr(L, name).argtypes = [ctypes.POINTER(OrCtx), _u32p, _u32p, ctypes.c_size_t]
        L.or_mont_mul_vec.argtypes = [ctypes.POINTER(OrCtx), _u32p, _u32p, _u32p, ctypes.c_size_t]
        L.or_mont_fma_vec.argtypes = [ctypes.POINTER(OrCtx), _u32p, _u32p, _u32p, _u32p,
                                      ctypes.c_size_t]
        L.or_mulmod_vec.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, ctypes.c_size_t]
        L.or_primitive_root.argtypes = [ctypes.c_uint32]
        L.or_primitive_root.restype = ctypes.c_uint32
        L.or_root_of_unity.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int]
        L.or_root_of_unity.restype = ctypes.c_uint32
        for name in ("or_dft", "or_ntt"):
            getattr(L, name).argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_size_t, ctypes.c_int]
            getattr(L, name).restype = ctypes.c_int
        L.or_polymul_schoolbook.argtypes = [ctypes.c_uint32, _u32p, ctypes.c_size_t, _u32p,
                                            ctypes.c_size_t, _u32p]
        L.or_polymul_ntt.argtypes = [ctypes.c_uint32, _u32p, ctypes.c_size_t, _u32p,
                                     ctypes.c_size_t, _u32p]
        L.or_polymul_ntt.restype = ctypes.c_int
        L.or_polymul_batch.argtypes = [_u32p, _u32p, _u64p, _u64p, _u32p, _u64p, _u64p, _u32p,
                                       _u64p, ctypes.c_size_t, ctypes.c_int]
        L.or_polymul_batch.restype = ctypes.c_int
        L.or_num_threads.restype = ctypes.c_int
        for name in ("or_tft", "or_itft"):
            getattr(L, name).argtypes = [ctypes.c_uint32, _u32p, ctypes.c_size_t, ctypes.c_int, _u32p]
            getattr(L, name).restype = ctypes.c_int
        L.or_polymul_tft.argtypes = [ctypes.c_uint32, _u32p, ctypes.c_size_t, _u32p, ctypes.c_size_t, _u32p]
        L.or_polymul_tft.restype = ctypes.c_int
        L.or_set_num_threads.argtypes = [ctypes.c_int]
        L.or_set_num_threads.restype = None
        _lib = L
    return _lib


def _u32(x):
    return np.ascontiguousarray(x, dtype=np.uint32)


def _ptr(a):
    return a.ctypes.data_as(_u32p if a.dtype == np.uint32 else _u64p)


def setup(p):
    """Montgomery constants for modulus p: P', R^-1, R mod P, R^2 mod P (Sec. 3.1)."""
    c = OrCtx()
    if lib().or_setup(p, ctypes.byref(c)) != 0:
        raise ValueError("oracle: modulus %r must be odd, 3 <= P < 2^31" % (p,))
    return c


def mulmod(a, b, p):
    return lib().or_mulmod(a, b, p)


def powmod(a, e, p):
    return lib().or_powmod(a, e, p)


def invmod(a, m):
    return lib().or_invmod(a, m)


def _vec1(fname, p, x):
    c = setup(p)
    x = _u32(x)
    out = np.empty_like(x)
    getattr(lib(), fname)(ctypes.byref(c), _ptr(x), _ptr(out), x.size)
    return out


def to_mont(p, x):
    """x R mod P elementwise."""
    return _vec1("or_to_mont_vec", p, x)


def from_mont(p, x):
    """x R^-1 mod P elementwise."""
    return _vec1("or_from_mont_vec", p, x)


def mont_mul(p, x, y):
    """x y R^-1 mod P elementwise: the value REDC(x, y) must return (Alg. 2)."""
    c = setup(p)
    x, y = _u32(x), _u32(y)
    assert x.shape == y.shape
    out = np.empty_like(x)
    lib().or_mont_mul_vec(ctypes.byref(c), _ptr(x), _ptr(y), _ptr(out), x.size)
    return out


def mont_fma(p, x, y, z):
    """(x y R^-1 + z) mod P elementwise."""
    c = setup(p)
    x, y, z = _u32(x), _u32(y), _u32(z)
    assert x.shape == y.shape == z.shape
    out = np.empty_like(x)
    lib().or_mont_fma_vec(ctypes.byref(c), _ptr(x), _ptr(y), _ptr(z), _ptr(out), x.size)
    return out


def mulmod_vec(p, x, y):
    """(x y) mod P elementwise."""
    x, y = _u32(x), _u32(y)
    out = np.empty_like(x)
    lib().or_mulmod_vec(p, _ptr(x), _ptr(y), _ptr(out), x.size)
    return out


def primitive_root(p):
    return lib().or_primitive_root(p)


def root_of_unity(p, n, inverse=False):
    w = lib().or_root_of_unity(p, n, int(bool(inverse)))
    if w == 0:
        raise ValueError("oracle: %d does not divide P - 1 = %d" % (n, p - 1))
    return w


def dft(p, x, inverse=False):
    """Direct O(N^2) DFT over Z_P, natural order; the inverse includes N^-1."""
    x = _u32(x)
    out = np.empty_like(x)
    if lib().or_dft(p, _ptr(x), _ptr(out), x.size, int(bool(inverse))) != 0:
        raise ValueError("oracle: no %d-th root of unity mod %d" % (x.size, p))
    return out


def ntt(p, x, inverse=False):
    """Recursive radix-2 NTT (same result as dft)."""
    x = _u32(x)
    out = np.empty_like(x)
    if lib().or_ntt(p, _ptr(x), _ptr(out), x.size, int(bool(inverse))) != 0:
        raise ValueError("oracle: bad NTT size %d mod %d" % (x.size, p))
    return out


def polymul_schoolbook(p, a, b):
    a, b = _u32(a), _u32(b)
    if a.size == 0 or b.size == 0:
        raise ValueError("oracle: empty operand")
    c = np.empty(a.size + b.size - 1, dtype=np.uint32)
    lib().or_polymul_schoolbook(p, _ptr(a), a.size, _ptr(b), b.size, _ptr(c))
    return c


def polymul_ntt(p, a, b):
    a, b = _u32(a), _u32(b)
    if a.size == 0 or b.size == 0:
        raise ValueError("oracle: empty operand")
    c = np.empty(a.size + b.size - 1, dtype=np.uint32)
    if lib().or_polymul_ntt(p, _ptr(a), a.size, _ptr(b), b.size, _ptr(c)) != 0:
        raise ValueError("oracle: product too long for P")
    return c


def tft(p, x, log2n):
    """Truncated Fourier transform (van der Hoeven): the first len(x) outputs,
    in bit-reversed order, of the size-2^log2n transform of x zero-padded."""
    x = _u32(x)
    out = np.empty_like(x)
    if lib().or_tft(p, _ptr(x), x.size, int(log2n), _ptr(out)) != 0:
        raise ValueError("oracle: bad TFT length %d for 2^%d mod %d" % (x.size, log2n, p))
    return out


def itft(p, y, log2n):
    """Inverse truncated Fourier transform: the x (len(y) entries) with tft(x) == y."""
    y = _u32(y)
    out = np.empty_like(y)
    if lib().or_itft(p, _ptr(y), y.size, int(log2n), _ptr(out)) != 0:
        raise ValueError("oracle: bad TFT length %d for 2^%d mod %d" % (y.size, log2n, p))
    return out


def polymul_tft(p, a, b):
    """a * b through TFTs of length len(a) + len(b) - 1."""
    a, b = _u32(a), _u32(b)
    if a.size == 0 or b.size == 0:
        raise ValueError("oracle: empty operand")
    c = np.empty(a.size + b.size - 1, dtype=np.uint32)
    if lib().or_polymul_tft(p, _ptr(a), a.size, _ptr(b), b.size, _ptr(c)) != 0:
        raise ValueError("oracle: product too long for P")
    return c


def polymul_batch(ps, a, a_off, la, b, b_off, lb, c_off, c_size, use_ntt=False):
    """Independent products in one call (OpenMP over products); returns c."""
    ps = _u32(ps)
    a, b = _u32(a), _u32(b)
    a_off, la, b_off, lb, c_off = (np.ascontiguousarray(v, dtype=np.uint64)
                                   for v in (a_off, la, b_off, lb, c_off))
    c = np.zeros(c_size, dtype=np.uint32)
    rc = lib().or_polymul_batch(_ptr(ps), _ptr(a), _ptr(a_off), _ptr(la), _ptr(b), _ptr(b_off),
                                _ptr(lb), _ptr(c), _ptr(c_off), ps.size, int(bool(use_ntt)))
    if rc != 0:
        raise ValueError("oracle: batch product failed")
    return c


def num_threads():
    return lib().or_num_threads()


class threads:
    """Context manager: the oracle's OpenMP loops use n threads inside (for
    timing it single-threaded), the previous count again after."""

    def __init__(self, n):
        self.n = int(n)

    def __enter__(self):
        self.prev = num_threads()
        lib().or_set_num_threads(self.n)
        return self

    def __exit__(self, *exc):
        lib().or_set_num_threads(self.prev)
        return False


__all__ = [n for n in dir() if not n.startswith("_")]
