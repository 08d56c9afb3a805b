"""ctypes binding over ``libmontgomery.so`` (the C ABI declared in include/mont.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  Tensors are torch CUDA tensors of dtype int32 or
uint32 holding residues in [0, P); the current torch stream of the tensor's
device is used unless a stream is given.  There is no CPU path: if the
library has not been built, every call raises.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmontgomery.so")

MONT_OK = 0
MONT_EINVAL = -1
MONT_ENOMEM = -2
MONT_ERANGE = -3
MONT_ETIMEOUT = -4
MONT_ECUDA = -5
MONT_EUNSUPPORTED = -6

_vp = ctypes.c_void_p
_sz = ctypes.c_size_t


class MontError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))


class MontCtx(ctypes.Structure):
    """Mirror of ``mont_ctx``: p, P' = -P^-1 mod 2^32, R mod P, R^2 mod P."""
    _fields_ = [("p", ctypes.c_uint32), ("p_prime", ctypes.c_uint32),
                ("r_mod_p", ctypes.c_uint32), ("r2_mod_p", ctypes.c_uint32)]

    def __repr__(self):
        return "MontCtx(p=%d, p_prime=%d, r_mod_p=%d, r2_mod_p=%d)" % (
            self.p, self.p_prime, self.r_mod_p, self.r2_mod_p)


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmontgomery.so is not built; run paper_1609_00999_gb300.build.build() "
                               "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    ctxp = ctypes.POINTER(MontCtx)
    L.mont_setup.argtypes = [ctypes.c_uint32, ctxp]
    L.mont_strerror.argtypes = [ctypes.c_int]
    L.mont_strerror.restype = ctypes.c_char_p
    L.to_mont.argtypes = [ctxp, _vp, _vp, _sz, _vp]
    L.from_mont.argtypes = [ctxp, _vp, _vp, _sz, _vp]
    L.mont_mul.argtypes = [ctxp, _vp, _vp, _vp, _sz, _vp]
    L.mont_fma.argtypes = [ctxp, _vp, _vp, _vp, _vp, _sz, _vp]
    L.barrett_mulmod.argtypes = [ctypes.c_uint32, _vp, _vp, _vp, _sz, _vp]
    L.fourier_redc_mul.argtypes = [ctxp, _vp, _vp, _vp, _sz, _vp]
    L.mont_check_residues.argtypes = [ctypes.c_uint32, _vp, _sz, _vp]
    L.mont_check_residues.restype = ctypes.c_int
    for name in ("mont_setup", "to_mont", "from_mont", "mont_mul", "mont_fma", "barrett_mulmod",
                 "fourier_redc_mul"):
        getattr(L, name).restype = ctypes.c_int
    _declare_ntt(L)


def _declare_ntt(L):
    L.ntt_plan_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_vp)]
    L.ntt_plan_create.restype = ctypes.c_int
    L.ntt_plan_destroy.argtypes = [_vp]
    L.ntt_plan_destroy.restype = None
    for name in ("ntt_fwd", "ntt_inv"):
        getattr(L, name).argtypes = [_vp, _vp, _sz, ctypes.c_int, _vp]
        getattr(L, name).restype = ctypes.c_int
    L.polymul.argtypes = [ctypes.c_uint32, _vp, _sz, _vp, _sz, _vp, _vp]
    L.polymul.restype = ctypes.c_int
    L.polymul_many.argtypes = [ctypes.c_uint32, _vp, _sz, _vp, _sz, _vp, _sz, _vp]
    L.polymul_many.restype = ctypes.c_int
    L.polymul_many_fourier.argtypes = [ctypes.c_uint32, _vp, _sz, _vp, _sz, _vp, _sz, _vp]
    L.polymul_many_fourier.restype = ctypes.c_int
    L.polymul_many_ws.argtypes = [ctypes.c_uint32, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _sz, _vp]
    L.polymul_many_ws.restype = ctypes.c_int
    L.polymul_workspace_bytes.argtypes = [_sz, _sz, _sz]
    L.polymul_workspace_bytes.restype = _sz
    L.polymul_noalloc.argtypes = [_vp, _vp, _sz, _vp, _sz, _vp, _vp]
    L.polymul_noalloc.restype = ctypes.c_int
    _declare_batch(L)
    _declare_server(L)
    L.mont_release_workspaces.argtypes = []
    L.mont_release_workspaces.restype = ctypes.c_int
    L.mont_int_probe.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp,
                                 ctypes.POINTER(ctypes.c_uint64), _vp]
    L.mont_int_probe.restype = ctypes.c_int


class PolymulDesc(ctypes.Structure):
    """Mirror of ``polymul_desc``."""
    _fields_ = [("a", _vp), ("b", _vp), ("c", _vp), ("la", ctypes.c_uint32), ("lb", ctypes.c_uint32),
                ("p", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class PolymulBatchConfig(ctypes.Structure):
    """Mirror of ``polymul_batch_config``."""
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("order", ctypes.c_int), ("kernel", ctypes.c_int),
                ("full_transforms", ctypes.c_int)]

    def __repr__(self):
        return "PolymulBatchConfig(ctas_per_sm=%d, order=%d, kernel=%d, full_transforms=%d)" % (
            self.ctas_per_sm, self.order, self.kernel, self.full_transforms)


def _declare_batch(L):
    vpp = ctypes.POINTER(_vp)
    L.polymul_batch_plan_create.argtypes = [ctypes.POINTER(PolymulDesc), _sz, vpp]
    L.polymul_batch_describe.argtypes = [ctypes.POINTER(PolymulDesc), _sz, ctypes.c_int, ctypes.c_int, _vp, _sz, _vp,
                                         ctypes.POINTER(_sz)]
    L.polymul_batch_describe.restype = ctypes.c_int
    L.polymul_batch_plan_destroy.argtypes = [_vp]
    L.polymul_batch_plan_destroy.restype = None
    L.polymul_batch_plan_workspace_bytes.argtypes = [_vp]
    L.polymul_batch_plan_workspace_bytes.restype = _sz
    L.polymul_batch_plan_get_config.argtypes = [_vp, ctypes.POINTER(PolymulBatchConfig)]
    L.polymul_batch_plan_set_config.argtypes = [_vp, ctypes.POINTER(PolymulBatchConfig)]
    L.polymul_batch_run.argtypes = [_vp, _vp]
    L.polymul_batch_run_graph.argtypes = [_vp, _vp]
    L.polymul_batch_status.argtypes = [_vp, _vp]
    L.polymul_batch_plan_tune.argtypes = [_vp, _vp, ctypes.c_int]
    L.polymul_batch_plan_set_wait_limit.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint64]
    L.polymul_batch_plan_inject_stall.argtypes = [_vp]
    L.polymul_batch.argtypes = [ctypes.POINTER(PolymulDesc), _sz, _vp, _sz, _vp]
    L.polymul_batch.restype = ctypes.c_int
    L.polymul_batch_workspace_bytes.argtypes = [ctypes.POINTER(PolymulDesc), _sz]
    L.polymul_batch_workspace_bytes.restype = _sz
    L.polymul_batch_check.argtypes = [_vp, _vp]
    L.polymul_batch_check.restype = ctypes.c_int
    for name in ("polymul_batch_plan_create", "polymul_batch_plan_get_config", "polymul_batch_plan_set_config",
                 "polymul_batch_run", "polymul_batch_run_graph", "polymul_batch_status", "polymul_batch_plan_tune",
                 "polymul_batch_plan_set_wait_limit", "polymul_batch_plan_inject_stall"):
        getattr(L, name).restype = ctypes.c_int


class MontServerStats(ctypes.Structure):
    """Mirror of ``mont_server_stats``."""
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "launched", "completed", "batches", "queued",
                                               "admitted_waiting", "in_flight", "bytes_in_use", "peak_bytes",
                                               "budget_bytes")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


def _declare_server(L):
    vpp = ctypes.POINTER(_vp)
    L.mont_server_create.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.c_int, ctypes.c_uint32, _sz,
                                     ctypes.c_int, _sz, vpp]
    L.mont_server_destroy.argtypes = [_vp]
    L.mont_server_destroy.restype = None
    L.mont_server_submit.argtypes = [_vp, _vp, _sz]
    L.mont_server_progress.argtypes = [_vp, _vp, _sz, ctypes.POINTER(_sz)]
    L.mont_server_get_stats.argtypes = [_vp, ctypes.POINTER(MontServerStats)]
    for name in ("mont_server_create", "mont_server_submit", "mont_server_progress", "mont_server_get_stats"):
        getattr(L, name).restype = ctypes.c_int


def strerror(code):
    try:
        return lib().mont_strerror(code).decode()
    except RuntimeError:
        return "error %d" % code


def _check(rc, what):
    if rc != MONT_OK:
        raise MontError(rc, what)


_U32_DTYPES = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())


def _dev_ptr(t, name):
    """Address of a CUDA tensor, or of a pinned host tensor (the kernels then
    read and write it in place over the CPU-GPU link, with no staging copy)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda and not t.is_pinned():
        raise ValueError("%s must be a CUDA tensor or a pinned host tensor" % name)
    if t.dtype not in _U32_DTYPES:
        raise TypeError("%s must be int32 or uint32 (got %s)" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t.data_ptr()


def _stream_handle(stream, device):
    if stream is None:
        if device is None or getattr(device, "type", "cuda") != "cuda":
            return torch.cuda.current_stream().cuda_stream
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def mont_setup(p):
    """Montgomery context for modulus p (host only)."""
    ctx = MontCtx()
    _check(lib().mont_setup(int(p), ctypes.byref(ctx)), "mont_setup(%r)" % (p,))
    return ctx


def _ctx(ctx):
    return ctx if isinstance(ctx, MontCtx) else mont_setup(ctx)


def _out_like(x, out):
    if out is None:
        return torch.empty_like(x)
    if out.numel() != x.numel():
        raise ValueError("out has %d elements, expected %d" % (out.numel(), x.numel()))
    return out


def to_mont(ctx, x, out=None, stream=None):
    """out = x R mod P (elementwise)."""
    ctx = _ctx(ctx)
    out = _out_like(x, out)
    _check(lib().to_mont(ctypes.byref(ctx), _dev_ptr(x, "x"), _dev_ptr(out, "out"), x.numel(),
                         _stream_handle(stream, x.device)), "to_mont")
    return out


def from_mont(ctx, x, out=None, stream=None):
    """out = x R^-1 mod P (elementwise)."""
    ctx = _ctx(ctx)
    out = _out_like(x, out)
    _check(lib().from_mont(ctypes.byref(ctx), _dev_ptr(x, "x"), _dev_ptr(out, "out"), x.numel(),
                           _stream_handle(stream, x.device)), "from_mont")
    return out


def mont_mul(ctx, a, b, out=None, stream=None):
    """out = REDC(a, b) = a b R^-1 mod P (elementwise, Alg. 2)."""
    ctx = _ctx(ctx)
    if a.numel() != b.numel():
        raise ValueError("a and b differ in size")
    out = _out_like(a, out)
    _check(lib().mont_mul(ctypes.byref(ctx), _dev_ptr(a, "a"), _dev_ptr(b, "b"), _dev_ptr(out, "out"),
                          a.numel(), _stream_handle(stream, a.device)), "mont_mul")
    return out


def mont_fma(ctx, a, b, c, out=None, stream=None):
    """out = (REDC(a, b) + c) mod P (elementwise)."""
    ctx = _ctx(ctx)
    if not (a.numel() == b.numel() == c.numel()):
        raise ValueError("a, b and c differ in size")
    out = _out_like(a, out)
    _check(lib().mont_fma(ctypes.byref(ctx), _dev_ptr(a, "a"), _dev_ptr(b, "b"), _dev_ptr(c, "c"),
                          _dev_ptr(out, "out"), a.numel(), _stream_handle(stream, a.device)), "mont_fma")
    return out


def barrett_mulmod(p, a, b, out=None, stream=None):
    """out = a b mod p on plain residues (Barrett reduction, Alg. 1)."""
    if a.numel() != b.numel():
        raise ValueError("a and b differ in size")
    out = _out_like(a, out)
    _check(lib().barrett_mulmod(int(p), _dev_ptr(a, "a"), _dev_ptr(b, "b"), _dev_ptr(out, "out"), a.numel(),
                                _stream_handle(stream, a.device)), "barrett_mulmod")
    return out


def fourier_redc_mul(ctx, a, b, out=None, stream=None):
    """out = a b R^-1 mod P by Montgomery reduction over a Fourier prime (Alg. 3; P < 2^30)."""
    ctx = _ctx(ctx)
    if a.numel() != b.numel():
        raise ValueError("a and b differ in size")
    out = _out_like(a, out)
    _check(lib().fourier_redc_mul(ctypes.byref(ctx), _dev_ptr(a, "a"), _dev_ptr(b, "b"), _dev_ptr(out, "out"),
                                  a.numel(), _stream_handle(stream, a.device)), "fourier_redc_mul")
    return out


def check_residues(p, x, stream=None):
    """True if every word of x lies in [0, p), False if some word is >= p
    (a synchronous device-side check of the inputs' precondition)."""
    rc = lib().mont_check_residues(int(p), _dev_ptr(x, "x"), x.numel(), _stream_handle(stream, x.device))
    if rc == MONT_ERANGE:
        return False
    _check(rc, "mont_check_residues")
    return True


NTT_BITREV = 1


class NttPlan:
    """Owner of an ``ntt_plan *`` (prime p, size 2^log2n, resident twiddles)."""

    def __init__(self, p, log2n):
        h = _vp()
        _check(lib().ntt_plan_create(int(p), int(log2n), ctypes.byref(h)), "ntt_plan_create(%r, %r)" % (p, log2n))
        self._h = h
        self.p = int(p)
        self.log2n = int(log2n)
        self.n = 1 << self.log2n

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ntt_plan_destroy(h)
            self._h = None


def ntt_plan_create(p, log2n):
    return NttPlan(p, log2n)


def _ntt(name, plan, data, flags, stream):
    if data.numel() % plan.n:
        raise ValueError("data size %d is not a multiple of N = %d" % (data.numel(), plan.n))
    _check(getattr(lib(), name)(plan.handle, _dev_ptr(data, "data"), data.numel() // plan.n, int(flags),
                                _stream_handle(stream, data.device)), name)
    return data


def ntt_fwd(plan, data, flags=0, stream=None):
    """In-place forward NTT of each row of N residues (natural order unless NTT_BITREV)."""
    return _ntt("ntt_fwd", plan, data, flags, stream)


def ntt_inv(plan, data, flags=0, stream=None):
    """In-place inverse NTT (with N^-1) of each row; input bit-reversed if NTT_BITREV."""
    return _ntt("ntt_inv", plan, data, flags, stream)


def polymul(p, a, b, out=None, stream=None):
    """c = a * b mod p for 1-D coefficient tensors; c has len(a) + len(b) - 1 entries."""
    lc = a.numel() + b.numel() - 1
    if out is None:
        out = torch.empty(max(lc, 0), dtype=a.dtype, device=a.device)
    elif out.numel() != lc:
        raise ValueError("out must have %d elements" % lc)
    _check(lib().polymul(int(p), _dev_ptr(a, "a"), a.numel(), _dev_ptr(b, "b"), b.numel(), _dev_ptr(out, "out"),
                         _stream_handle(stream, a.device)), "polymul")
    return out


def polymul_many(p, a, b, out=None, stream=None):
    """Row-wise products of a [count][la] and b [count][lb] -> [count][la + lb - 1]."""
    if a.dim() != 2 or b.dim() != 2 or a.shape[0] != b.shape[0]:
        raise ValueError("a and b must be [count][la] and [count][lb]")
    count, la = a.shape
    lb = b.shape[1]
    lc = la + lb - 1
    if out is None:
        out = torch.empty((count, lc), dtype=a.dtype, device=a.device)
    elif out.numel() != count * lc:
        raise ValueError("out must have %d elements" % (count * lc))
    _check(lib().polymul_many(int(p), _dev_ptr(a, "a"), la, _dev_ptr(b, "b"), lb, _dev_ptr(out, "out"), count,
                              _stream_handle(stream, a.device)), "polymul_many")
    return out


def polymul_many_fourier(p, a, b, out=None, stream=None):
    """polymul_many with the FourierREDC (Alg. 3) twiddle multiply: Fourier
    primes below 2^30 with 2n >= 32, N <= 2^14; identical results."""
    if a.dim() != 2 or b.dim() != 2 or a.shape[0] != b.shape[0]:
        raise ValueError("a and b must be [count][la] and [count][lb]")
    count, la = a.shape
    lb = b.shape[1]
    lc = la + lb - 1
    if out is None:
        out = torch.empty((count, lc), dtype=a.dtype, device=a.device)
    elif out.numel() != count * lc:
        raise ValueError("out must have %d elements" % (count * lc))
    _check(lib().polymul_many_fourier(int(p), _dev_ptr(a, "a"), la, _dev_ptr(b, "b"), lb, _dev_ptr(out, "out"),
                                      count, _stream_handle(stream, a.device)), "polymul_many_fourier")
    return out


def polymul_workspace_bytes(la, lb, count=1):
    """Scratch bytes polymul_many_ws needs (0 when N <= 2^14)."""
    return int(lib().polymul_workspace_bytes(int(la), int(lb), int(count)))


def polymul_many_ws(p, a, b, workspace, out=None, stream=None):
    """polymul_many with a caller-owned scratch tensor (any dtype, CUDA, contiguous)."""
    if a.dim() != 2 or b.dim() != 2 or a.shape[0] != b.shape[0]:
        raise ValueError("a and b must be [count][la] and [count][lb]")
    count, la = a.shape
    lb = b.shape[1]
    lc = la + lb - 1
    if out is None:
        out = torch.empty((count, lc), dtype=a.dtype, device=a.device)
    elif out.numel() != count * lc:
        raise ValueError("out must have %d elements" % (count * lc))
    ws_ptr = workspace.data_ptr() if workspace is not None else None
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().polymul_many_ws(int(p), _dev_ptr(a, "a"), la, _dev_ptr(b, "b"), lb, _dev_ptr(out, "out"), count,
                                 ws_ptr, ws_bytes, _stream_handle(stream, a.device)), "polymul_many_ws")
    return out


def mont_release_workspaces():
    _check(lib().mont_release_workspaces(), "mont_release_workspaces")


def polymul_noalloc(plan, a, b, out=None, stream=None):
    """polymul through the entry point that allocates nothing: twiddles from
    `plan` (same prime, 2^plan.log2n >= len(a) + len(b) - 1), scratch from the
    library's fixed device array (len(a) + len(b) - 1 <= 2^18).  `out` must be
    given by callers that cannot let torch allocate."""
    lc = a.numel() + b.numel() - 1
    if out is None:
        out = torch.empty(max(lc, 0), dtype=a.dtype, device=a.device)
    elif out.numel() != lc:
        raise ValueError("out must have %d elements" % lc)
    _check(lib().polymul_noalloc(plan.handle, _dev_ptr(a, "a"), a.numel(), _dev_ptr(b, "b"), b.numel(),
                                 _dev_ptr(out, "out"), _stream_handle(stream, a.device)), "polymul_noalloc")
    return out


PROBE_KINDS = {"imad": 0, "imad_hi": 1, "imad_wide": 2, "iadd3": 3, "redc": 4, "ct": 5, "ct_one": 6,
               "ct_first": 7, "gs": 8, "gs_one": 9}


def int_probe(kind, p, iterations, sink, ctas_per_sm=0, stream=None):
    """Queues one integer-pipe probe launch (``mont_int_probe``) of the named
    kind (a key of PROBE_KINDS) and returns the number of operations it
    performs; `sink` is a CUDA int32 tensor of at least one element."""
    ops = ctypes.c_uint64(0)
    _check(lib().mont_int_probe(PROBE_KINDS[kind], int(p), int(iterations), int(ctas_per_sm), _dev_ptr(sink, "sink"),
                                ctypes.byref(ops), _stream_handle(stream, sink.device)), "mont_int_probe")
    return int(ops.value)


def _check_packed_bounds(na, a_off, la, nb, b_off, lb, nc, c_off):
    """ValueError unless, for every product i, a[a_off[i]:][:la[i]],
    b[b_off[i]:][:lb[i]] and c[c_off[i]:][:la[i] + lb[i] - 1] lie inside
    tensors of na, nb and nc words (lengths >= 1, offsets >= 0)."""
    import numpy as np
    cols = [np.asarray(x, dtype=np.int64).reshape(-1) for x in (a_off, la, b_off, lb, c_off)]
    if len({x.size for x in cols}) != 1:
        raise ValueError("offset and length sequences differ in size")
    ao, la_, bo, lb_, co = cols
    if ao.size == 0:
        return
    if (la_ < 1).any() or (lb_ < 1).any():
        raise ValueError("product lengths must be >= 1")
    if (ao < 0).any() or (bo < 0).any() or (co < 0).any():
        raise ValueError("offsets must be >= 0")
    for name, end, n in (("a", ao + la_, na), ("b", bo + lb_, nb), ("c", co + la_ + lb_ - 1, nc)):
        bad = np.flatnonzero(end > n)
        if bad.size:
            raise ValueError("product %d: %s slice ends at %d, beyond the %d-word tensor"
                             % (bad[0], name, end[bad[0]], n))


class PolymulBatchPlan:
    """Owner of a ``polymul_batch_plan *``: an uneven batch of products run by
    one persistent kernel launch (or a CUDA graph replay of it)."""

    def __init__(self, descs, keepalive=()):
        arr = (PolymulDesc * max(1, len(descs)))()
        for i, d in enumerate(descs):
            arr[i] = d
        h = _vp()
        _check(lib().polymul_batch_plan_create(arr, len(descs), ctypes.byref(h)), "polymul_batch_plan_create")
        self._h = h
        self._keep = tuple(keepalive)
        self.count = len(descs)

    @classmethod
    def from_packed(cls, primes, a, a_off, la, b, b_off, lb, c, c_off):
        """Products packed back to back: product i uses a[a_off[i]:][:la[i]] etc.
        (a, b, c int32/uint32 CUDA tensors; offsets and lengths host sequences).
        Every slice must lie inside its tensor: the kernel sees raw addresses."""
        _check_packed_bounds(a.numel(), a_off, la, b.numel(), b_off, lb, c.numel(), c_off)
        pa, pb, pc = _dev_ptr(a, "a"), _dev_ptr(b, "b"), _dev_ptr(c, "c")
        descs = [PolymulDesc(pa + 4 * int(ao), pb + 4 * int(bo), pc + 4 * int(co), int(x), int(y), int(p), 0)
                 for p, ao, x, bo, y, co in zip(primes, a_off, la, b_off, lb, c_off)]
        return cls(descs, keepalive=(a, b, c))

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self):
        return int(lib().polymul_batch_plan_workspace_bytes(self._h))

    @property
    def config(self):
        c = PolymulBatchConfig()
        _check(lib().polymul_batch_plan_get_config(self._h, ctypes.byref(c)), "polymul_batch_plan_get_config")
        return c

    @config.setter
    def config(self, cfg):
        _check(lib().polymul_batch_plan_set_config(self._h, ctypes.byref(cfg)), "polymul_batch_plan_set_config")

    def run(self, stream=None, device=None):
        _check(lib().polymul_batch_run(self._h, _stream_handle(stream, device)), "polymul_batch_run")

    def run_graph(self, stream=None, device=None):
        _check(lib().polymul_batch_run_graph(self._h, _stream_handle(stream, device)), "polymul_batch_run_graph")

    def status(self, stream=None, device=None):
        """Synchronise and return MONT_OK or MONT_ETIMEOUT (no exception)."""
        return lib().polymul_batch_status(self._h, _stream_handle(stream, device))

    def tune(self, trials=3, stream=None, device=None):
        rc = lib().polymul_batch_plan_tune(self._h, _stream_handle(stream, device), int(trials))
        _check(rc, "polymul_batch_plan_tune")
        return self.config

    def set_wait_limit(self, iterations, nanoseconds):
        _check(lib().polymul_batch_plan_set_wait_limit(self._h, int(iterations), int(nanoseconds)),
               "polymul_batch_plan_set_wait_limit")

    def inject_stall(self):
        _check(lib().polymul_batch_plan_inject_stall(self._h), "polymul_batch_plan_inject_stall")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.polymul_batch_plan_destroy(h)
            self._h = None


def polymul_batch_plan_create(descs, keepalive=()):
    return PolymulBatchPlan(descs, keepalive)


def polymul_batch_describe(descs, order, full_transforms=0):
    """Host only: (jobs [n][4] uint32: kind, log2 N, product, index;
    prods [count][4] uint32: log2 N, column tiles, rows computed, truncated
    transform flag) of the job list the batch kernel runs for these
    descriptors in job order `order`."""
    import numpy as np
    arr = (PolymulDesc * max(1, len(descs)))()
    for i, d in enumerate(descs):
        arr[i] = d
    n = _sz(0)
    _check(lib().polymul_batch_describe(arr, len(descs), int(order), int(full_transforms), None, 0, None,
                                        ctypes.byref(n)), "polymul_batch_describe")
    jobs = np.zeros((max(1, n.value), 4), dtype=np.uint32)
    prods = np.zeros((max(1, len(descs)), 4), dtype=np.uint32)
    _check(lib().polymul_batch_describe(arr, len(descs), int(order), int(full_transforms), jobs.ctypes.data, n.value,
                                        prods.ctypes.data, ctypes.byref(n)), "polymul_batch_describe")
    return jobs[:n.value], prods[:len(descs)]


def _desc_array(descs):
    arr = (PolymulDesc * max(1, len(descs)))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def polymul_batch_workspace_bytes(descs):
    """Workspace bytes polymul_batch needs for these descriptors (host only;
    0 for an empty list or invalid descriptors)."""
    return int(lib().polymul_batch_workspace_bytes(_desc_array(descs), len(descs)))


def polymul_batch(descs, workspace, stream=None):
    """One-shot uneven batch: PolymulDesc list, caller-owned CUDA workspace
    tensor (any dtype, contiguous) of at least polymul_batch_workspace_bytes
    bytes.  Queues the work and returns; polymul_batch_check reports waits
    that expired."""
    if not isinstance(workspace, torch.Tensor) or not workspace.is_cuda or not workspace.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().polymul_batch(_desc_array(descs), len(descs), workspace.data_ptr(), nbytes,
                               _stream_handle(stream, workspace.device)), "polymul_batch")


def polymul_batch_check(workspace, stream=None):
    """Synchronises the stream; MONT_OK or MONT_ETIMEOUT for the last
    polymul_batch run on this workspace."""
    return int(lib().polymul_batch_check(workspace.data_ptr(), _stream_handle(stream, workspace.device)))


# numpy mirrors of mont_request / mont_completion (48 and 16 bytes)
def request_dtype():
    import numpy as np
    return np.dtype([("a", np.uint64), ("b", np.uint64), ("c", np.uint64), ("la", np.uint32), ("lb", np.uint32),
                     ("p", np.uint32), ("reserved", np.uint32), ("id", np.uint64)])


def completion_dtype():
    import numpy as np
    return np.dtype([("id", np.uint64), ("status", np.int32), ("reserved", np.int32)])


def _check_request_array(reqs, start, stop):
    """The library reads mont_request structs straight from the array's
    memory: it must be a C-contiguous 1-D array of request_dtype() and
    0 <= start <= stop <= len(reqs)."""
    import numpy as np
    if not isinstance(reqs, np.ndarray) or reqs.dtype != request_dtype():
        raise TypeError("reqs must be a numpy array of request_dtype()")
    if reqs.ndim != 1 or not reqs.flags.c_contiguous:
        raise ValueError("reqs must be a 1-D C-contiguous array")
    if not (0 <= start <= stop <= len(reqs)):
        raise ValueError("need 0 <= start <= stop <= len(reqs), got %r, %r" % (start, stop))


class MontServer:
    """Owner of a ``mont_server *`` (continuous-batching request server)."""

    def __init__(self, primes, max_log2n, budget_bytes, slots=4, max_batch_coeffs=1 << 25):
        import numpy as np
        arr = (ctypes.c_uint32 * len(primes))(*[int(p) for p in primes])
        h = _vp()
        _check(lib().mont_server_create(arr, len(primes), int(max_log2n), int(budget_bytes), int(slots),
                                        int(max_batch_coeffs), ctypes.byref(h)), "mont_server_create")
        self._h = h
        self._done = np.zeros(1 << 16, dtype=completion_dtype())

    def submit(self, reqs, start=0, stop=None):
        """Queue requests [start, stop) of a request_dtype() array."""
        stop = len(reqs) if stop is None else stop
        _check_request_array(reqs, start, stop)
        if stop > start:
            ptr = reqs.ctypes.data + start * reqs.dtype.itemsize
            _check(lib().mont_server_submit(self._h, ptr, stop - start), "mont_server_submit")

    def progress(self):
        """One non-blocking step; returns the completions (a completion_dtype() array view)."""
        n = _sz()
        _check(lib().mont_server_progress(self._h, self._done.ctypes.data, len(self._done), ctypes.byref(n)),
               "mont_server_progress")
        return self._done[:n.value]

    def stats(self):
        st = MontServerStats()
        _check(lib().mont_server_get_stats(self._h, ctypes.byref(st)), "mont_server_get_stats")
        return st.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.mont_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()
