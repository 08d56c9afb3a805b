"""polymul_noalloc, the entry point that allocates nothing, against polymul.

Callers that cannot call cudaMalloc (graph capture, a framework that owns the
device memory, latency-critical paths) use polymul_noalloc, whose scratch is
a fixed array in the library's device memory.  Its results must equal the
allocating polymul's, bit for bit, on two calls in a row (the second call
must not see anything left over from the first).  This file is collected
last so that a run stopping at its first failure has run everything else.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("p", synth.PRIMES)
def test_noalloc_matches_polymul_twice(m, p):
    import torch
    plan = m.ntt_plan_create(p, 18)          # set-up: tables for every N <= 2^18
    shapes = [(100000, 31073), (70001, 50000), (3000, 1000), (1 << 17, (1 << 17) + 1)]
    for call in range(2):                    # two calls in a row per shape, different inputs
        for la, lb in shapes:
            a = synth.residues(la, p, 500, call, la, 0)
            b = synth.residues(lb, p, 500, call, la, 1)
            da, db = to_dev(a), to_dev(b)
            out = torch.empty(la + lb - 1, dtype=torch.int32, device="cuda")
            m.polymul_noalloc(plan, da, db, out=out)
            ref = m.polymul(p, da, db)
            assert np.array_equal(to_host(out), to_host(ref)), (call, la, lb)


def test_noalloc_rejects_beyond_maximum(m):
    import torch
    p = synth.P1
    plan = m.ntt_plan_create(p, 19)
    a = to_dev(np.ones((1 << 17) + 2, dtype=np.uint32))
    b = to_dev(np.ones(1 << 17, dtype=np.uint32))
    out = torch.empty(a.numel() + b.numel() - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(m.MontError) as e:            # la + lb - 1 = 2^18 + 1 > 2^18
        m.polymul_noalloc(plan, a, b, out=out)
    assert e.value.code == m.MONT_ERANGE
    small_plan = m.ntt_plan_create(p, 10)
    a2, b2 = to_dev(np.ones(600, dtype=np.uint32)), to_dev(np.ones(600, dtype=np.uint32))
    with pytest.raises(m.MontError) as e:            # plan's tables shorter than N = 2^11
        m.polymul_noalloc(small_plan, a2, b2, out=torch.empty(1199, dtype=torch.int32, device="cuda"))
    assert e.value.code == m.MONT_ERANGE
