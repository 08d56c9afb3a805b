"""polymul_noalloc, the entry point that allocates nothing, against the CPU
oracle and against polymul.

Callers that cannot call cudaMalloc (graph capture, a framework that owns the
device memory, latency-critical paths) use polymul_noalloc, whose scratch is
a fixed array in the library's device memory.  Its results must equal the
oracle's product and the allocating polymul's, bit for bit, on two calls in a
row (the second call must not see anything left over from the first), and
the second round of calls must leave the device's free memory and torch's
reserved memory unchanged.  This file is collected last so that a run
stopping at its first failure has run everything else.
"""
import numpy as np
import pytest

import oracle
from paper_1609_00999_gb300 import synth

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

# N = 2^12 (one fused kernel), 2^15 and 2^16 (the scratch array's column /
# row splits below its maximum), 2^17 and 2^18 (the largest it accepts).
SHAPES = [(3000, 1000), (20000, 10000), (40000, 20000), (70001, 50000), (100000, 31073),
          (1 << 17, (1 << 17) + 1)]


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
def test_noalloc_matches_oracle_and_polymul_twice(m, p):
    import torch
    plan = m.ntt_plan_create(p, 18)          # set-up: tables for every N <= 2^18
    host, dev, outs = {}, {}, {}
    for call in range(2):                    # two calls in a row per shape, different inputs
        for la, lb in SHAPES:
            a = synth.residues(la, p, 500, call, la, 0)
            b = synth.residues(lb, p, 500, call, la, 1)
            host[call, la, lb] = (a, b)
            dev[call, la, lb] = (to_dev(a), to_dev(b))
            outs[call, la, lb] = torch.full((la + lb - 1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:                        # the first round loaded every kernel the second one runs
            free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        for la, lb in SHAPES:
            da, db = dev[call, la, lb]
            m.polymul_noalloc(plan, da, db, out=outs[call, la, lb])
        torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0
    for call in range(2):
        for la, lb in SHAPES:
            a, b = host[call, la, lb]
            got = to_host(outs[call, la, lb])
            assert np.array_equal(got, oracle.polymul_ntt(p, a, b)), (call, la, lb)
            da, db = dev[call, la, lb]
            assert np.array_equal(got, to_host(m.polymul(p, da, db))), (call, la, lb)


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
