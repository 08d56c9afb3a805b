"""The continuous-batching request server: a Poisson stream of products of
mixed sizes and primes under a small device-memory budget.  Every result must
be bit-exact equal to the same product computed alone and to the oracle's
product, whatever else was in flight with it."""
import numpy as np
import pytest

import oracle
from paper_1609_00999_gb300 import serve, synth

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


def stream_case(n=400, lo=1 << 8, hi=1 << 15, rate=20000.0, seed=700):
    lens = synth.loguniform_lengths(n, lo, hi, seed, 0)
    primes = synth.choose_primes(n, seed, 1)
    arrivals = synth.poisson_arrivals(n, rate, seed, 2)
    wl = synth.UnevenBatch(primes, lens, lens, (seed,))
    return wl, arrivals


STREAMS = {
    # lengths up to 2^15 under a 24 MiB budget: admission waits, many small batches
    "small": dict(case=dict(n=400, hi=1 << 15, rate=20000.0), max_log2n=16, budget=24 << 20, cap=1 << 17),
    # the serving workload's full length range, L up to 2^20 (N up to 2^21)
    "full_range": dict(case=dict(n=160, hi=1 << 20, rate=2000.0, seed=701), max_log2n=21, budget=256 << 20,
                       cap=1 << 22),
    # 2,000 requests over the serving workload's length range [2^8, 2^20] with
    # the benchmark's batch cap (2^24 coefficients) under a 1 GiB budget
    "full_range_2000": dict(case=dict(n=2000, hi=1 << 20, rate=4000.0, seed=702), max_log2n=21, budget=1 << 30,
                            cap=1 << 24),
}


@pytest.mark.parametrize("name", sorted(STREAMS))
def test_stream_results_equal_alone(m, name):
    import torch
    cfg = STREAMS[name]
    wl, arrivals = stream_case(**cfg["case"])
    da, db = to_dev(wl.a), to_dev(wl.b)
    host_a = torch.from_numpy(wl.a.view(np.int32)).pin_memory()       # half the requests read host memory
    hc = torch.full((wl.c_size,), -1, dtype=torch.int32).pin_memory()
    n = len(wl)
    use_host = (np.arange(n) % 2) == 1
    a_ptrs = np.where(use_host, host_a.data_ptr(), da.data_ptr()) + 4 * wl.a_off.astype(np.int64)
    reqs = serve.make_requests(wl.primes, wl.la, wl.lb, a_ptrs,
                               db.data_ptr() + 4 * wl.b_off.astype(np.int64),
                               hc.data_ptr() + 4 * wl.c_off.astype(np.int64))
    budget = cfg["budget"]
    server = m.MontServer(synth.PRIMES, cfg["max_log2n"], budget, slots=3, max_batch_coeffs=cfg["cap"])
    lat, status, makespan = serve.run_stream(server, reqs, arrivals)
    st = server.stats()
    server.close()
    assert np.all(status == m.MONT_OK)
    assert np.all(np.isfinite(lat)) and np.all(lat >= 0)
    assert st["completed"] == n and st["peak_bytes"] <= budget and st["batches"] > 3
    got = hc.numpy().view(np.uint32)
    for i in range(n):
        ao, la = int(wl.a_off[i]), int(wl.la[i])
        bo, lb = int(wl.b_off[i]), int(wl.lb[i])
        co = int(wl.c_off[i])
        alone = to_host(m.polymul(int(wl.primes[i]), da[ao:ao + la], db[bo:bo + lb]))
        assert np.array_equal(got[co:co + la + lb - 1], alone), i
    # every request against the oracle (one OpenMP call over all products)
    ref = oracle.polymul_batch(wl.primes, wl.a, wl.a_off, wl.la, wl.b, wl.b_off, wl.lb, wl.c_off, wl.c_size,
                               use_ntt=True)
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, "%d wrong words; first in request %d" % (
        bad.size, int(np.searchsorted(wl.c_off.astype(np.int64), bad[0], side="right") - 1) if bad.size else -1)


def test_server_rejects_bad_requests(m):
    import torch
    d = to_dev(np.ones(1 << 12, dtype=np.uint32))
    out = torch.zeros(1 << 13, dtype=torch.int32, device="cuda")
    server = m.MontServer([synth.P1], 14, 1 << 15, slots=1)
    big = serve.make_requests([synth.P1], [4096], [4096], [d.data_ptr()], [d.data_ptr()], [out.data_ptr()])
    with pytest.raises(m.MontError) as e:           # needs 64 KiB, more than the whole 32 KiB budget
        server.submit(big)
    assert e.value.code == m.MONT_ERANGE
    other = serve.make_requests([synth.P2], [8], [8], [d.data_ptr()], [d.data_ptr()], [out.data_ptr()])
    with pytest.raises(m.MontError) as e:           # prime not served
        server.submit(other)
    assert e.value.code == m.MONT_EINVAL
    ok = serve.make_requests([synth.P1], [100], [50], [d.data_ptr()], [d.data_ptr()], [out.data_ptr()])
    lat, status, _ = serve.run_stream(server, ok, np.zeros(1))
    server.close()
    assert status[0] == m.MONT_OK
    assert np.array_equal(to_host(out)[:149], oracle.polymul_schoolbook(synth.P1, np.ones(100, np.uint32),
                                                                        np.ones(50, np.uint32)))
