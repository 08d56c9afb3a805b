"""Polynomial-multiplication sections of the benchmark (imported by bench.py).

* uniform batch: 4096 products of length-2048 polynomials mod 2013265921
  (N = 4096), one fused kernel; L2 flushed between timed launches because
  the 64 MiB of operands fit in L2;
* uneven batch: 10,000 products, lengths log-uniform in [2^6, 2^16], primes
  uniform from the three Fourier primes, one persistent launch replayed from
  a CUDA graph after autotuning, against one launch per product;
* serve: 50,000 requests, lengths log-uniform in [2^8, 2^20], mixed primes,
  Poisson arrivals at 0.8 x the measured saturated request rate, a 16 GB
  device-memory budget; throughput and p50/p99 latency.

Gcoef/s counts input coefficients (la + lb per product) per second.
Integer roofline: the path runs on the two 32-bit integer pipes of each SM
sub-partition (ALU and FMA-heavy, 16 lanes each), i.e. 128 integer lane-ops
per SM per clock; 32x32->64 multiplies (IMAD.WIDE / IMAD.HI) issue at half
rate and count 2.  The algorithmic lane-ops of a product are counted per
butterfly from the method (see int_ops_polymul).
"""
import time

import numpy as np

from paper_1609_00999_gb300 import serve, synth

SMS = 152
INT_LANES_PER_SM_CLK = 128


def int_peak_ops(sm_mhz):
    return SMS * INT_LANES_PER_SM_CLK * sm_mhz * 1e6


def int_ops_polymul(n, la, lb):
    """Algorithmic integer lane-ops of one product of size n (power of two).

    Non-trivial CT butterfly: REDC (wide mul 2, mul.lo 1, wide mul-add 2) +
    conditional subtract 1 + add/subtract with their conditional subtracts 4
    = 10; non-trivial GS butterfly: 9 (its difference feeds REDC unreduced);
    butterfly with twiddle 1 (block 0 of every level, n - 1 per transform): 4;
    stand-alone REDC (pointwise product, scaling of b): 6."""
    levels = n.bit_length() - 1
    bfly = (n // 2) * levels
    trivial = n - 1
    nontrivial = bfly - trivial
    fwd = 2 * (10 * nontrivial + 4 * trivial)
    inv = 9 * nontrivial + 4 * trivial
    return fwd + inv + 6 * n + 6 * lb


def batch_hbm_bytes(n, la, lb):
    """Algorithmic HBM bytes of one product of size n in the batch kernel:
    operands in and result out; products of 2^14 and 2^15 (whole-product
    jobs) also read their operands once per row (2 or 4 rows) and pass their
    product rows through scratch (n words out and back); larger ones move
    2n words of forward scratch out and back, n words of product rows out
    and back."""
    lc = la + lb - 1
    io = 4 * (la + lb + lc)
    if n <= 1 << 13:
        return io
    if n <= 1 << 15:
        rows = n >> 13
        return io + 4 * (rows - 1) * (la + lb) + 4 * 2 * n
    return io + 4 * (2 * 2 * n + 2 * n)


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def uniform_batch(m, torch, peaks, steps=20, warmup=3, cpu=True):
    import oracle
    p, a, b = synth.batch_uniform()
    count, L = a.shape
    n = 1 << (2 * L - 1).bit_length()
    da = torch.from_numpy(a.view(np.int32)).cuda()
    db = torch.from_numpy(b.view(np.int32)).cuda()
    out = torch.empty((count, 2 * L - 1), dtype=torch.int32, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")   # 256 MiB > L2
    for _ in range(warmup):
        m.polymul_many(p, da, db, out=out)
    torch.cuda.synchronize()
    # All steps are queued before one synchronize, so the GPU never waits for
    # the host between the start event and the launch it brackets.
    evs = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = _events(torch)
        e0.record()
        m.polymul_many(p, da, db, out=out)
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))
    coeffs = count * 2 * L
    ops = count * int_ops_polymul(n, L, L)
    peak = int_peak_ops(peaks["sm_max_mhz"])
    hbm_bytes = count * (2 * L + 2 * L - 1) * 4
    res = {"workload": "4096 products, la = lb = 2048, P = 2013265921, N = 4096 (one fused kernel)",
           "value": coeffs / ms / 1e6, "unit": "Gcoef/s", "ms": ms, "steps": steps, "warmup": warmup,
           "l2": "flushed (256 MiB write) before every timed launch", "gpu_launches": steps,
           "roofline": {"bound": "alu", "kernel": "k_polymul<12, RedAlg2>", "achieved": ops / (ms / 1e3) / 1e12,
                        "peak": peak / 1e12, "unit": "Tops/s (integer lane-ops)", "frac": ops / (ms / 1e3) / peak,
                        "peak_source": "derived: 152 SMs x 128 int lanes/clk x %.0f MHz" % peaks["sm_max_mhz"],
                        "algorithmic_ops": ops, "traffic": None},
           "hbm_at_pass_count": {"passes": 1, "bytes": hbm_bytes, "achieved_gbs": hbm_bytes / (ms / 1e3) / 1e9,
                                 "peak_gbs": peaks["hbm_gbs"],
                                 "frac": hbm_bytes / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}}
    # parity spot check on this run's output (full parity lives in the tests)
    got = out[:4].cpu().numpy().view(np.uint32)
    for i in range(4):
        assert np.array_equal(got[i], oracle.polymul_ntt(p, a[i], b[i])), "polymul parity spot check failed"
    if cpu:
        off = np.arange(count, dtype=np.uint64) * L
        lens = np.full(count, L, dtype=np.uint64)
        t0 = time.perf_counter()
        oracle.polymul_batch(np.full(count, p, dtype=np.uint32), a.ravel(), off, lens, b.ravel(), off, lens,
                             np.arange(count, dtype=np.uint64) * (2 * L - 1), count * (2 * L - 1), use_ntt=True)
        t = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": coeffs / t / 1e9, "unit": "Gcoef/s", "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "all 4096 products (oracle radix-2 NTT, OpenMP over products)"}
    del flush
    return res


def int_ops_ntt(n, inverse):
    """Algorithmic integer lane-ops of one transform of size n (as in
    int_ops_polymul): non-trivial CT butterflies 10, GS 9, twiddle-1
    butterflies 4, plus the inverse's N^-1 scaling REDC (6) per element."""
    levels = n.bit_length() - 1
    trivial = n - 1
    nontrivial = (n // 2) * levels - trivial
    if inverse:
        return 9 * nontrivial + 4 * trivial + 6 * n
    return 10 * nontrivial + 4 * trivial


def roundtrip_small(m, torch, steps=200, warmup=10):
    """The 65,536-pair correctness workload as a latency figure: to_mont of a
    and b, mont_mul, from_mont (four launches per step), P1."""
    import oracle
    p, a, b = synth.elementwise_small()
    ctx = m.mont_setup(p)
    da = torch.from_numpy(a.view(np.int32)).cuda()
    db = torch.from_numpy(b.view(np.int32)).cuda()
    am, bm, pm, out = (torch.empty_like(da) for _ in range(4))

    def step():
        m.to_mont(ctx, da, out=am)
        m.to_mont(ctx, db, out=bm)
        m.mont_mul(ctx, am, bm, out=pm)
        m.from_mont(ctx, pm, out=out)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    e1.synchronize()
    us = e0.elapsed_time(e1) / steps * 1e3
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.mulmod_vec(p, a, b)), "round trip parity failed"
    return {"workload": "65,536 pairs mod P1: to_mont a, to_mont b, mont_mul, from_mont (4 launches)",
            "us_per_step": us, "us_per_launch": us / 4, "steps": steps, "warmup": warmup,
            "l2": "operands (256 KiB each) stay in L2: a latency figure", "gpu_launches": 4 * steps,
            "parity": "bit-exact against (a b) mod P"}


def ntt_transforms(m, torch, peaks, steps=10, warmup=3):
    """Stand-alone ntt_fwd / ntt_inv (natural order in and out): 4096 rows of
    N = 4096 (one fused kernel each, L2 flushed before every launch) and 16
    rows of N = 2^20 (column / row kernels and the bit-reversal), P1."""
    import oracle
    p = synth.P1
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    peak = int_peak_ops(peaks["sm_max_mhz"])
    res = {}
    for rows, logn in ((4096, 12), (16, 20)):
        n = 1 << logn
        x = synth.residues(rows * n, p, 900, logn).reshape(rows, n)
        plan = m.ntt_plan_create(p, logn)
        d = torch.from_numpy(x.view(np.int32)).cuda()
        for _ in range(warmup):
            m.ntt_fwd(plan, d)
            m.ntt_inv(plan, d)
        torch.cuda.synchronize()
        evs = {"fwd": [], "inv": []}
        for _ in range(steps):
            for k, f in (("fwd", m.ntt_fwd), ("inv", m.ntt_inv)):
                flush.fill_(1)
                e0, e1 = _events(torch)
                e0.record()
                f(plan, d)
                e1.record()
                evs[k].append((e0, e1))
        torch.cuda.synchronize()
        assert torch.equal(d.cpu(), torch.from_numpy(x.view(np.int32))), "inverse(forward(x)) != x"
        m.ntt_fwd(plan, d)
        got0 = d[0].cpu().numpy().view(np.uint32)
        assert np.array_equal(got0, oracle.ntt(p, x[0])), "ntt parity spot check failed"
        r = {"rows": rows, "n": n, "unit": "Gcoef/s", "l2": "flushed (256 MiB write) before every launch",
             "gpu_launches_per_call": 1 if logn <= 14 else 3}
        for k in ("fwd", "inv"):
            ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs[k]]))
            ops = rows * int_ops_ntt(n, k == "inv")
            r[k] = {"ms": ms, "value": rows * n / ms / 1e6,
                    "roofline": {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e12, "peak": peak / 1e12,
                                 "unit": "Tops/s (integer lane-ops)", "frac": ops / (ms / 1e3) / peak},
                    "hbm_gbs_at_pass_count": rows * n * 8 * (1 if logn <= 14 else 3) / (ms / 1e3) / 1e9}
        res["N%d_x%d" % (n, rows)] = r
        del d
    del flush
    res["parity"] = "inverse(forward(x)) == x for every row; row 0 of the forward equal to the oracle's NTT"
    return res


def reductions_elementwise(m, torch, peaks, log2n=28, steps=10, warmup=3):
    """The three reductions of Sec. 3.1 on the same vectors: Barrett (Alg. 1,
    a b mod P on plain residues), REDC (Alg. 2) and FourierREDC (Alg. 3, a b
    R^-1 mod P), 2^log2n residues per operand mod P2 = 469762049 (the prime
    all three accept).  12 B per element: HBM-bound unless a reduction's
    arithmetic outruns the memory time."""
    import oracle
    p = synth.P2
    n = 1 << log2n
    a = synth.residues(n, p, 950, 0)
    b = synth.residues(n, p, 950, 1)
    da = torch.from_numpy(a.view(np.int32)).cuda()
    db = torch.from_numpy(b.view(np.int32)).cuda()
    out = torch.empty_like(da)
    ctx = m.mont_setup(p)
    fns = {"alg1_barrett": lambda: m.barrett_mulmod(p, da, db, out=out),
           "alg2_redc": lambda: m.mont_mul(ctx, da, db, out=out),
           "alg3_fourier_redc": lambda: m.fourier_redc_mul(ctx, da, db, out=out)}
    res = {"workload": "2^%d residues per operand mod 469762049, one elementwise multiply" % log2n,
           "unit": "Gmulmod/s", "steps": steps, "warmup": warmup, "bytes_per_element": 12,
           "l2": "operands larger than L2; no flush", "gpu_launches": steps * len(fns)}
    sample = np.arange(0, n, 4099, dtype=np.int64)
    for k, f in fns.items():
        for _ in range(warmup):
            f()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(steps):
            f()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        got = out.cpu().numpy().view(np.uint32)[sample]
        ref = (oracle.mulmod_vec(p, a[sample], b[sample]) if k == "alg1_barrett"
               else oracle.mont_mul(p, a[sample], b[sample]))
        assert np.array_equal(got, ref), "%s parity spot check failed" % k
        res[k] = {"ms": ms, "value": n / ms / 1e6, "hbm_gbs": 12 * n / ms / 1e6,
                  "hbm_frac": 12 * n / ms / 1e6 / peaks["hbm_gbs"]}
    del da, db, out
    torch.cuda.empty_cache()
    return res


def reduction_ab(m, torch, steps=20, warmup=3):
    """Alg. 2 (REDC) against Alg. 3 (FourierREDC) as the twiddle, scaling and
    pointwise multiply of the same fused kernels: 4096 products of
    length-2048 polynomials mod P2 = 469762049 (Alg. 3 needs P < 2^30), L2
    flushed before every launch, launches alternating between the two."""
    import oracle
    p, a, b = synth.batch_uniform(p=synth.P2)
    count, L = a.shape
    da = torch.from_numpy(a.view(np.int32)).cuda()
    db = torch.from_numpy(b.view(np.int32)).cuda()
    out = {k: torch.empty((count, 2 * L - 1), dtype=torch.int32, device="cuda") for k in ("alg2", "alg3")}
    fns = {"alg2": m.polymul_many, "alg3": m.polymul_many_fourier}
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    for _ in range(warmup):
        for k, f in fns.items():
            f(p, da, db, out=out[k])
    torch.cuda.synchronize()
    evs = {k: [] for k in fns}
    for _ in range(steps):
        for k, f in fns.items():
            flush.fill_(1)
            e0, e1 = _events(torch)
            e0.record()
            f(p, da, db, out=out[k])
            e1.record()
            evs[k].append((e0, e1))
    torch.cuda.synchronize()
    assert torch.equal(out["alg2"], out["alg3"]), "Alg. 2 and Alg. 3 products differ"
    got = out["alg3"][:2].cpu().numpy().view(np.uint32)
    for i in range(2):
        assert np.array_equal(got[i], oracle.polymul_ntt(p, a[i], b[i])), "Alg. 3 parity spot check failed"
    res = {"workload": "4096 products, la = lb = 2048, P = 469762049, N = 4096 (one fused kernel each)",
           "unit": "Gcoef/s", "steps": steps, "warmup": warmup, "l2": "flushed (256 MiB write) before every launch",
           "gpu_launches": 2 * steps}
    for k in fns:
        ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs[k]]))
        res[k] = {"ms": ms, "value": count * 2 * L / ms / 1e6,
                  "kernel": "k_polymul<12, %s>" % ("RedAlg2" if k == "alg2" else "RedAlg3")}
    res["alg3_over_alg2_time"] = res["alg3"]["ms"] / res["alg2"]["ms"]
    del flush
    return res


def uneven_batch(m, torch, peaks, steps=10, warmup=3, cpu=True, per_product=True, config=None):
    import oracle
    wl = synth.batch_uneven()
    da = torch.from_numpy(wl.a.view(np.int32)).cuda()
    db = torch.from_numpy(wl.b.view(np.int32)).cuda()
    dc = torch.empty(wl.c_size, dtype=torch.int32, device="cuda")
    plan = m.PolymulBatchPlan.from_packed(wl.primes, da, wl.a_off, wl.la, db, wl.b_off, wl.lb, dc, wl.c_off)
    t0 = time.perf_counter()
    if config is None:
        cfg = plan.tune(trials=2)
    else:                                   # fixed launch shape (ctas_per_sm, order, kernel): no tuning launches
        plan.config = m.PolymulBatchConfig(*config)
        cfg = plan.config
    tune_s = time.perf_counter() - t0
    for _ in range(warmup):
        plan.run_graph()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(steps):
        plan.run_graph()
    e1.record()
    e1.synchronize()
    assert plan.status() == m.MONT_OK
    ms = e0.elapsed_time(e1) / steps
    coeffs = float((wl.la + wl.lb).sum())
    ns = [1 << int(lc - 1).bit_length() for lc in (wl.la + wl.lb - 1)]
    ops = float(sum(int_ops_polymul(n, int(la), int(lb)) for n, la, lb in zip(ns, wl.la, wl.lb)))
    peak = int_peak_ops(peaks["sm_max_mhz"])
    hbm = float(sum(batch_hbm_bytes(n, int(la), int(lb)) for n, la, lb in zip(ns, wl.la, wl.lb)))
    res = {"workload": "10,000 products, L log-uniform in [2^6, 2^16], primes uniform from "
                       "{2013265921, 469762049, 754974721}, N padded to powers of two",
           "value": coeffs / ms / 1e6, "unit": "Gcoef/s", "ms": ms, "steps": steps, "warmup": warmup,
           "launch": "one persistent kernel per batch, replayed from a CUDA graph",
           "tuned_config": {"ctas_per_sm": cfg.ctas_per_sm, "order": cfg.order, "kernel": cfg.kernel,
                            "tuned": config is None}, "tune_s": tune_s,
           "workspace_bytes": plan.workspace_bytes(), "l2": "operands + scratch (2.4 GB) larger than L2",
           "gpu_launches": steps,
           "roofline": {"bound": "alu", "kernel": "k_polymul_batch", "achieved": ops / (ms / 1e3) / 1e12,
                        "peak": peak / 1e12, "unit": "Tops/s (integer lane-ops)", "frac": ops / (ms / 1e3) / peak,
                        "algorithmic_ops": ops, "traffic": None},
           "hbm_at_pass_count": {"bytes": hbm, "achieved_gbs": hbm / (ms / 1e3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
                                 "frac": hbm / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                 "passes": "one for N <= 2^13; operands, results and the product rows' scratch "
                                           "round trip for 2^14 and 2^15 (operands read 2 or 4 times); "
                                           "three passes through 2N words of scratch above"}}
    # spot check a few products against the oracle
    got = dc.cpu().numpy().view(np.uint32)
    for i in (0, 1, 9999):
        ao, la, bo, lb, co = (int(wl.a_off[i]), int(wl.la[i]), int(wl.b_off[i]), int(wl.lb[i]), int(wl.c_off[i]))
        ref = oracle.polymul_ntt(int(wl.primes[i]), wl.a[ao:ao + la], wl.b[bo:bo + lb])
        assert np.array_equal(got[co:co + la + lb - 1], ref), "batch parity spot check failed"
    if per_product:
        L = m.lib()
        stream = torch.cuda.current_stream().cuda_stream
        pa, pb, pc = da.data_ptr(), db.data_ptr(), dc.data_ptr()
        args = [(int(wl.primes[i]), pa + 4 * int(wl.a_off[i]), int(wl.la[i]), pb + 4 * int(wl.b_off[i]),
                 int(wl.lb[i]), pc + 4 * int(wl.c_off[i])) for i in range(len(wl))]
        for a_ in args[:50]:
            L.polymul(a_[0], a_[1], a_[2], a_[3], a_[4], a_[5], stream)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        w0 = time.perf_counter()
        e0.record()
        for a_ in args:
            rc = L.polymul(a_[0], a_[1], a_[2], a_[3], a_[4], a_[5], stream)
            assert rc == 0
        e1.record()
        e1.synchronize()
        wall = time.perf_counter() - w0
        one_ms = e0.elapsed_time(e1)
        res["one_launch_per_product"] = {"value": coeffs / one_ms / 1e6, "unit": "Gcoef/s", "ms": one_ms,
                                         "host_wall_ms": wall * 1e3,
                                         "note": "polymul() per product on one stream, same products"}
        res["batched_over_per_product"] = one_ms / ms
    if cpu:
        k = 1000
        t0 = time.perf_counter()
        oracle.polymul_batch(wl.primes[:k], wl.a, wl.a_off[:k], wl.la[:k], wl.b, wl.b_off[:k], wl.lb[:k],
                             wl.c_off[:k], int(wl.c_off[k - 1] + wl.la[k - 1] + wl.lb[k - 1] - 1), use_ntt=True)
        t = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": float((wl.la[:k] + wl.lb[:k]).sum()) / t / 1e9, "unit": "Gcoef/s",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "first 1000 of the 10,000 products (oracle radix-2 NTT, OpenMP)"}
    del plan
    return res


def serve_stream(m, torch, n=50000, budget=16 << 30, slots=4, batch_coeffs=1 << 24, load=0.8, pool_log2=24,
                 ring_words=1 << 30):
    lens = synth.loguniform_lengths(n, 1 << 8, 1 << 20, synth.SEED_SERVE, 0)
    primes = synth.choose_primes(n, synth.SEED_SERVE, 1)
    pool_n = 1 << pool_log2
    pools = {}
    for i, p in enumerate(synth.PRIMES):
        pools[p] = torch.from_numpy(synth.residues(pool_n, p, synth.SEED_SERVE, 10 + i).view(np.int32)).pin_memory()
    g = synth.rng(synth.SEED_SERVE, 3)
    off_a = (g.random(n) * (pool_n - lens + 1)).astype(np.int64)
    off_b = (g.random(n) * (pool_n - lens + 1)).astype(np.int64)
    base = np.array([pools[int(p)].data_ptr() for p in primes], dtype=np.int64)
    ring_t = torch.empty(ring_words, dtype=torch.int32).pin_memory()
    coeffs = float(2 * lens.sum())

    def make():
        return serve.make_requests(primes, lens, lens, base + 4 * off_a, base + 4 * off_b, np.zeros(n, np.int64))

    server = m.MontServer(synth.PRIMES, 21, budget, slots=slots, max_batch_coeffs=batch_coeffs)
    # warm-up: a short closed-loop burst
    warm = make()[:500]
    serve.run_stream(server, warm, np.zeros(len(warm)), ring=serve.HostRing(ring_t.data_ptr(), ring_words))
    # saturation: every request arrives at t = 0
    lat_s, st_s, mk_s = serve.run_stream(server, make(), np.zeros(n),
                                         ring=serve.HostRing(ring_t.data_ptr(), ring_words))
    rate_sat = n / mk_s
    lam = load * rate_sat
    arrivals = synth.poisson_arrivals(n, lam, synth.SEED_SERVE, 2)
    lat, st, mk = serve.run_stream(server, make(), arrivals, ring=serve.HostRing(ring_t.data_ptr(), ring_words))
    stats = server.stats()
    server.close()
    assert np.all(st == 0) and np.all(st_s == 0), "serve: a request failed"
    summ = serve.latency_summary(lat)
    return {"workload": "50,000 requests, L log-uniform in [2^8, 2^20], primes uniform from the three Fourier "
                        "primes, Poisson arrivals; operands from a seeded pinned host pool, results copied back",
            "value": coeffs / mk / 1e9, "unit": "Gcoef/s", "requests_per_s": n / mk, "makespan_s": mk,
            "lambda_per_s": lam, "load": load, "saturated": {"requests_per_s": rate_sat, "Gcoef_s": coeffs / mk_s / 1e9,
                                                              **serve.latency_summary(lat_s)},
            **summ, "budget_bytes": budget, "slots": slots, "max_batch_coeffs": batch_coeffs,
            "batches": stats["batches"], "peak_bytes": stats["peak_bytes"],
            "latency": "host clock, arrival (scheduled) to completion reported by mont_server_progress"}
