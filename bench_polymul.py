"""Polynomial-multiplication sections of the benchmark (imported by bench.py).

* integer-pipe probes: the measured ceiling of each operation the transforms
  run (single instruction forms, REDC, the NTT butterflies as the kernels
  inline them), timed with CUDA events;
* uniform batch: 4096 products of length-2048 polynomials mod 2013265921
  (N = 4096), one fused kernel; L2 flushed between timed launches because
  the 64 MiB of operands fit in L2;
* uneven batch: 10,000 products, lengths log-uniform in [2^6, 2^16], primes
  uniform from the three Fourier primes, one persistent launch replayed from
  a CUDA graph after autotuning, against one launch per product;
* serve: 50,000 requests, lengths log-uniform in [2^8, 2^20], mixed primes,
  Poisson arrivals at 0.5, 0.8, 1.0 and 1.2 x the measured saturated request
  rate, a 16 GB device-memory budget; throughput and p50/p99 latency.

Gcoef/s counts input coefficients (la + lb per product) per second.

Integer roofline.  The work of a product is counted per operation class:
Cooley-Tukey butterflies with a twiddle, with twiddle 1, and with twiddle 1
on reduced inputs (level 0), Gentleman-Sande butterflies with a twiddle and
with twiddle 1, and stand-alone REDCs (pointwise product, scaling).  The
probes measure each class's throughput on the device; the floor of a
workload is the sum over classes of count / throughput, and `frac` is that
floor over the kernel's measured time.  `achieved` and `peak` are expressed
in integer lane-ops (int_ops_polymul: wide multiplies count 2) so that they
compare with the nominal 128 lane-ops per SM per clock (`derived_peak`).
"""
import hashlib
import json
import os
import time

import numpy as np

from paper_1609_00999_gb300 import serve, synth

ROOT = os.path.dirname(os.path.abspath(__file__))
SMS = 152
INT_LANES_PER_SM_CLK = 128
PROBE_ORDER = ("imad", "imad_hi", "imad_wide", "iadd3", "redc", "ct", "ct_one", "ct_first", "gs", "gs_one")
OP_CLASSES = ("ct", "ct_one", "ct_first", "gs", "gs_one", "redc")
# Kernels (= HBM passes over the data) of a natural-order stand-alone
# transform above 2^14: column kernel, row kernel, bit reversal.
NTT_LARGE_PASSES = 3


def int_peak_ops(sm_mhz, sms=SMS):
    return sms * INT_LANES_PER_SM_CLK * sm_mhz * 1e6


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


def op_counts_polymul(n, lb):
    """Operations of one product of size n by class: two forward transforms
    (level 0 all in block 0: n/2 butterflies on reduced inputs; block 0 of
    levels 1 .. K-1: n/2 - 1 with twiddle 1; the rest with a twiddle), one
    inverse (n - 1 with twiddle 1), n pointwise REDCs and lb scaling REDCs
    of b.  n = 1: the two REDCs only."""
    if n == 1:
        return {"redc": 2}
    k = n.bit_length() - 1
    nontrivial = (n // 2) * k - (n - 1)
    return {"ct": 2 * nontrivial, "ct_first": 2 * (n // 2), "ct_one": 2 * (n // 2 - 1), "gs": nontrivial,
            "gs_one": n - 1, "redc": n + lb}


def op_counts_ntt(n, inverse):
    """Operations of one stand-alone transform of size n by class (the
    inverse adds its N^-1 scaling REDC per element)."""
    k = n.bit_length() - 1
    nontrivial = (n // 2) * k - (n - 1)
    if inverse:
        return {"gs": nontrivial, "gs_one": n - 1, "redc": n}
    return {"ct": nontrivial, "ct_first": n // 2, "ct_one": n // 2 - 1}


def add_counts(total, counts, times=1):
    for key, v in counts.items():
        total[key] = total.get(key, 0) + times * v
    return total


def floor_seconds(counts, rates):
    """Time the counted operations need at the probes' measured throughputs."""
    return sum(v / rates[key] for key, v in counts.items() if v)


def source_digest(paths):
    h = hashlib.sha256()
    for pth in paths:
        with open(os.path.join(ROOT, pth), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_ncu(kernel_key):
    """The committed ncu record of a kernel (profiles/ncu_traffic.json), or
    None when any of its source files changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)[kernel_key]
        if rec.get("source_digest") != source_digest(rec["sources"]):
            return None
        return rec
    except Exception:
        return None


def recorded_traffic(kernel_key, units):
    """DRAM bytes per launch from the committed ncu record, scaled to `units`
    (the record's unit: elements or products per launch), or None."""
    rec = recorded_ncu(kernel_key)
    if rec is None:
        return None
    return rec["dram_bytes_per_launch"] * units / rec["units_per_launch"]


def int_roofline(kernel, ops, counts, ms, peaks, traffic_units=None):
    """roofline object of an integer-bound kernel: `ops` lane-ops (and
    `counts` operations by class) in `ms` milliseconds.  The peak is the
    probes' measured ceiling for this mix when the probe section ran,
    otherwise the nominal lane count."""
    secs = ms / 1e3
    derived = int_peak_ops(peaks["sm_max_mhz"], peaks.get("sms", SMS))
    rates = peaks.get("probe_rates")
    rec = recorded_ncu(kernel)
    out = {"bound": "alu", "kernel": kernel, "achieved": ops / secs / 1e12, "unit": "Tops/s (integer lane-ops)",
           "algorithmic_ops": ops, "op_counts": counts,
           "derived_peak": derived / 1e12, "frac_of_derived": ops / secs / derived,
           "traffic": recorded_traffic(kernel, traffic_units) if traffic_units is not None else None}
    if rates:
        floor = floor_seconds(counts, rates)
        out.update(peak=ops / floor / 1e12, frac=floor / secs, floor_ms=floor * 1e3,
                   peak_source="measured: integer-pipe probes (mont_int_probe) weighted by this workload's "
                               "butterfly and REDC counts")
    else:
        out.update(peak=derived / 1e12, frac=ops / secs / derived,
                   peak_source="derived: %d SMs x 128 int lanes/clk x %.0f MHz (probes not run)"
                               % (peaks.get("sms", SMS), peaks["sm_max_mhz"]))
    if rec is not None and "fma_heavy_busy" in rec:
        out["ncu_fma_heavy_busy"] = rec["fma_heavy_busy"]
    return out


def int_probes(m, torch, p=None, target_ms=2.0, steps=5, warmup=2):
    """Throughput of every probe kind of mont_int_probe (operations per
    second over the whole GPU): a short launch sizes the iteration count to
    about target_ms, then `steps` launches are timed one by one with CUDA
    events and the median kept."""
    p = p or synth.P1
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    res = {}
    for kind in PROBE_ORDER:
        it = 32
        e0, e1 = _events(torch)
        e0.record()
        m.int_probe(kind, p, it, sink)
        e1.record()
        e1.synchronize()
        it = max(1, int(it * target_ms / max(e0.elapsed_time(e1), 1e-3)))
        for _ in range(warmup):
            ops = m.int_probe(kind, p, it, sink)
        evs = []
        for _ in range(steps):
            e0, e1 = _events(torch)
            e0.record()
            ops = m.int_probe(kind, p, it, sink)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = float(np.median([a.elapsed_time(b) for a, b in evs]))
        res[kind] = {"ops_per_s": ops / (ms / 1e3), "ms": ms, "iterations": it, "ops_per_launch": ops}
    return {"workload": "register-only chains: 8 per thread, 256-thread CTAs, as many per SM as fit; p = %d" % p,
            "unit": "operations per second (instructions, REDCs or butterflies)", "steps": steps,
            "gpu_launches": len(PROBE_ORDER) * (steps + warmup + 1), "kinds": res}


def probe_per_sm_clock(section, sm_mhz, sms):
    """Adds each probe's operations per SM per clock at the sampled SM clock."""
    for v in section["kinds"].values():
        v["per_sm_per_clk"] = v["ops_per_s"] / (sms * sm_mhz * 1e6)
    section["sm_mhz"] = sm_mhz
    section["sms"] = sms
    return section


ROW_LOG = 13   # rows of 2^13 in the batch kernel's split products


def tft_rows(n, lc):
    """Rows of 2^13 a batch product of size n computes when it runs as a
    row-granular truncated transform (the batch builder's rule: 2 <= log2 n -
    13 <= 4 and ceil(lc / 2^13) leaves rows unused), else None."""
    k1 = n.bit_length() - 1 - ROW_LOG
    if 2 <= k1 <= 4:
        need = -(-lc // (1 << ROW_LOG))
        if need < (1 << k1):
            return need
    return None


def skipped_row_ops(n, rows):
    """(operation counts, lane-ops) of the rows a truncated product does not
    compute: per row, the forward row levels of both operands and the
    inverse row levels (13 levels of 2^12 butterflies, all with a twiddle in
    rows 1 and up) and its 2^13 pointwise REDCs."""
    skipped = (n >> ROW_LOG) - rows
    per = (1 << (ROW_LOG - 1)) * ROW_LOG
    counts = {"ct": -2 * per * skipped, "gs": -per * skipped, "redc": -(1 << ROW_LOG) * skipped}
    return counts, -skipped * ((2 * 10 + 9) * per + 6 * (1 << ROW_LOG))


def batch_hbm_bytes(n, la, lb, rows=None):
    """Algorithmic HBM bytes of one product of size n in the batch kernel:
    operands in and result out; products of 2^14 and 2^15 (whole-product
    jobs) also read their operands once per row (2 or 4 rows) and pass their
    product rows through scratch (n words out and back); larger ones move
    2n words of forward scratch out and back, n words of product rows out
    and back.  A truncated product computing `rows` rows of 2^13 moves the
    scratch of those rows only."""
    lc = la + lb - 1
    io = 4 * (la + lb + lc)
    if n <= 1 << 13:
        return io
    if rows is None:
        rows = n >> 13
    if n <= 1 << 15:
        return io + 4 * (rows - 1) * (la + lb) + 4 * 2 * (rows << 13)
    return io + 4 * 6 * (rows << 13)


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
    counts = add_counts({}, op_counts_polymul(n, L), count)
    hbm_bytes = count * (2 * L + 2 * L - 1) * 4
    res = {"workload": "4096 products, la = lb = 2048, P = 2013265921, N = 4096 (one fused kernel)",
           "value": coeffs / ms / 1e6, "unit": "Gcoef/s", "ms": ms, "steps": steps, "warmup": warmup,
           "l2": "flushed (256 MiB write) before every timed launch", "gpu_launches": steps,
           "roofline": int_roofline("k_polymul<12, RedAlg2>", ops, counts, ms, peaks, traffic_units=count),
           "hbm_at_pass_count": {"passes": 1, "bytes": hbm_bytes, "achieved_gbs": hbm_bytes / (ms / 1e3) / 1e9,
                                 "peak_gbs": peaks["hbm_gbs"],
                                 "frac": hbm_bytes / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}}
    got = out.cpu().numpy().view(np.uint32)
    if cpu:
        # The CPU baseline computes every product of the workload; its result
        # is also the parity check of every output word of this run.
        off = np.arange(count, dtype=np.uint64) * L
        lens = np.full(count, L, dtype=np.uint64)
        t0 = time.perf_counter()
        ref = oracle.polymul_batch(np.full(count, p, dtype=np.uint32), a.ravel(), off, lens, b.ravel(), off, lens,
                                   np.arange(count, dtype=np.uint64) * (2 * L - 1), count * (2 * L - 1),
                                   use_ntt=True)
        t = time.perf_counter() - t0
        assert np.array_equal(got.ravel(), ref), "polymul parity check failed"
        res["parity"] = "every output word of all 4096 products equal to the oracle's"
        res["cpu_baseline"] = {"value": coeffs / t / 1e9, "unit": "Gcoef/s", "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "all 4096 products (oracle radix-2 NTT, OpenMP over products)"}
    else:
        for i in range(4):
            assert np.array_equal(got[i], oracle.polymul_ntt(p, a[i], b[i])), "polymul parity spot check failed"
        res["parity"] = "first 4 products equal to the oracle's"
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
        passes = 1 if logn <= 14 else NTT_LARGE_PASSES
        r = {"rows": rows, "n": n, "unit": "Gcoef/s", "l2": "flushed (256 MiB write) before every launch",
             "gpu_launches_per_call": passes, "hbm_passes": passes}
        for k in ("fwd", "inv"):
            ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs[k]]))
            ops = rows * int_ops_ntt(n, k == "inv")
            counts = add_counts({}, op_counts_ntt(n, k == "inv"), rows)
            kern = ("k_ntt_%s<%d>" % (k, logn)) if logn <= 14 else "ntt_%s 2^%d (column, row kernels)" % (k, logn)
            r[k] = {"ms": ms, "value": rows * n / ms / 1e6,
                    "roofline": int_roofline(kern, ops, counts, ms, peaks, traffic_units=rows),
                    "hbm_gbs_at_pass_count": rows * n * 8 * passes / (ms / 1e3) / 1e9}
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
    """The 10,000-product uneven workload in one persistent launch replayed
    from a CUDA graph: tuned (truncated transforms on, the default), then the
    same launch shape with every product padded to its full transform."""
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

    def timed():
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
        return e0.elapsed_time(e1) / steps

    ms = timed()
    got = dc.cpu().numpy().view(np.uint32)
    c_full = m.PolymulBatchConfig(cfg.ctas_per_sm, cfg.order, cfg.kernel, 1)
    plan.config = c_full
    dc.fill_(-1)
    ms_full = timed()
    got_full = dc.cpu().numpy().view(np.uint32)
    plan.config = cfg
    coeffs = float((wl.la + wl.lb).sum())
    lcs = (wl.la + wl.lb - 1).astype(np.int64)
    ns = [1 << int(lc - 1).bit_length() for lc in lcs]

    def work(truncated):
        ops, hbm, counts = 0.0, 0.0, {}
        for n, la, lb, lc in zip(ns, wl.la, wl.lb, lcs):
            rows = tft_rows(n, int(lc)) if truncated else None
            add_counts(counts, op_counts_polymul(n, int(lb)))
            ops += int_ops_polymul(n, int(la), int(lb))
            if rows is not None:
                c_skip, ops_skip = skipped_row_ops(n, rows)
                add_counts(counts, c_skip)
                ops += ops_skip
            hbm += batch_hbm_bytes(n, int(la), int(lb), rows)
        return ops, hbm, counts

    # The persistent kernel (kernel 0, 1) or the phased form (kernel 2: one
    # kernel per job kind, their traffic recorded together per batch).
    kern = "batch_phased" if cfg.kernel == 2 else "k_polymul_batch"

    def figures(t_ms, truncated):
        ops, hbm, counts = work(truncated)
        return {"ms": t_ms, "value": coeffs / t_ms / 1e6, "unit": "Gcoef/s",
                "roofline": int_roofline(kern, ops, counts, t_ms, peaks,
                                         traffic_units=len(wl) if truncated else None),
                "hbm_at_pass_count": {"bytes": hbm, "achieved_gbs": hbm / (t_ms / 1e3) / 1e9,
                                      "peak_gbs": peaks["hbm_gbs"],
                                      "frac": hbm / (t_ms / 1e3) / 1e9 / peaks["hbm_gbs"]}}

    # Kernels one run launches: the persistent kernel, or the phased form's
    # kernel per small-product size plus its three column / row kernels.
    small_sizes = {n for n in ns if n <= 1 << 13}
    kernels_per_run = len(small_sizes) + 3 if cfg.kernel == 2 else 1
    tft = figures(ms, True)
    full = figures(ms_full, False)
    n_trunc = sum(1 for n, lc in zip(ns, lcs) if tft_rows(n, int(lc)) is not None)
    res = {"workload": "10,000 products, L log-uniform in [2^6, 2^16], primes uniform from "
                       "{2013265921, 469762049, 754974721}, N padded to powers of two",
           "value": tft["value"], "unit": "Gcoef/s", "ms": ms, "steps": steps, "warmup": warmup,
           "launch": ("phased form: one kernel per job kind (small products by size, whole products, forward "
                      "columns, rows, output columns) on three branches of one CUDA graph"
                      if cfg.kernel == 2 else "one persistent kernel per batch, replayed from a CUDA graph"),
           "tuned_config": {"ctas_per_sm": cfg.ctas_per_sm, "order": cfg.order, "kernel": cfg.kernel,
                            "full_transforms": cfg.full_transforms, "tuned": config is None}, "tune_s": tune_s,
           "workspace_bytes": plan.workspace_bytes(), "l2": "operands + scratch (2.4 GB) larger than L2",
           "gpu_launches": 2 * (steps + warmup) * kernels_per_run, "kernels_per_run": kernels_per_run,
           "roofline": tft["roofline"],
           "hbm_at_pass_count": dict(tft["hbm_at_pass_count"],
                                     passes="one for N <= 2^13; operands, results and the product rows' scratch "
                                            "round trip for 2^14 and 2^15 (operands read once per row); three "
                                            "passes through the scratch of the rows computed above"),
           "truncated_products": n_trunc,
           "full_transforms": dict(full, note="same launch shape, every product padded to its full power-of-two "
                                              "transform (polymul_batch_config.full_transforms = 1)"),
           "full_over_truncated_time": ms_full / ms}
    if not cpu:
        for i in (0, 1, 9999):
            ao, la, bo, lb, co = (int(wl.a_off[i]), int(wl.la[i]), int(wl.b_off[i]), int(wl.lb[i]), int(wl.c_off[i]))
            ref = oracle.polymul_ntt(int(wl.primes[i]), wl.a[ao:ao + la], wl.b[bo:bo + lb])
            assert np.array_equal(got[co:co + la + lb - 1], ref), "batch parity spot check failed"
            assert np.array_equal(got_full[co:co + la + lb - 1], ref), "batch parity spot check failed"
        res["parity"] = "products 0, 1 and 9999 (truncated and full transforms) equal to the oracle's"
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
        # The CPU baseline computes all 10,000 products; its result is also
        # the parity check of every output word of both batch variants.
        t0 = time.perf_counter()
        ref = oracle.polymul_batch(wl.primes, wl.a, wl.a_off, wl.la, wl.b, wl.b_off, wl.lb, wl.c_off, wl.c_size,
                                   use_ntt=True)
        t = time.perf_counter() - t0
        assert np.array_equal(got[:wl.c_size], ref), "batch parity check failed (truncated transforms)"
        assert np.array_equal(got_full[:wl.c_size], ref), "batch parity check failed (full transforms)"
        res["parity"] = ("every output word of all 10,000 products equal to the oracle's, with truncated and "
                         "with full transforms")
        res["cpu_baseline"] = {"value": coeffs / t / 1e9, "unit": "Gcoef/s",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "all 10,000 products (oracle radix-2 NTT, OpenMP over products)"}
    del plan
    return res


def check_served(reqs, lens, primes, pools, off_a, off_b, ring_t, ring_words, load, sample=12, seed=17,
                 scan=20000):
    """Results of the last requests of a served stream that are still in the
    result ring when it ends, against the oracle: a request's result is
    intact if no later request's region (the placements the run recorded in
    reqs["c"]) overlaps it.  Among the intact ones of the last `scan`
    requests, `sample` drawn at random plus the last one are checked."""
    import bisect
    import oracle
    lc = 2 * lens.astype(np.int64) - 1
    base = ring_t.data_ptr()
    starts, ends = [], []            # union of the later requests' regions, disjoint, sorted
    intact = []
    for i in range(len(lc) - 1, max(-1, len(lc) - 1 - scan), -1):
        a = (int(reqs["c"][i]) - base) // 4
        b = a + int(lc[i])
        k = bisect.bisect_right(starts, a)
        hit = (k > 0 and ends[k - 1] > a) or (k < len(starts) and starts[k] < b)
        if not hit:
            intact.append(i)
        # merge [a, b) into the union
        lo = bisect.bisect_left(ends, a)
        hi = bisect.bisect_right(starts, b)
        if lo < hi:
            a, b = min(a, starts[lo]), max(b, ends[hi - 1])
        starts[lo:hi] = [a]
        ends[lo:hi] = [b]
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(intact, size=min(sample, len(intact)), replace=False).tolist()) if intact else set()
    pick.add(len(lc) - 1)
    ring = ring_t.numpy().view(np.uint32)
    for i in sorted(pick):
        p = int(primes[i])
        pool = pools[p].numpy().view(np.uint32)
        a = pool[off_a[i]:off_a[i] + lens[i]]
        b = pool[off_b[i]:off_b[i] + lens[i]]
        start = (int(reqs["c"][i]) - base) // 4
        got = ring[start:start + int(lc[i])]
        assert np.array_equal(got, oracle.polymul_ntt(p, a, b)), "serve parity failed for request %d" % i
    return ("%d of the %d intact results among the last %d requests of the load-%.1f stream, every output word "
            "equal to the oracle's" % (len(pick), len(intact), min(scan, len(lc)), load))


def serve_stream(m, torch, n=50000, budget=16 << 30, slots=4, batch_coeffs=1 << 24, loads=(0.5, 0.8, 1.0, 1.2),
                 headline_load=0.8, pool_log2=24, ring_words=1 << 30):
    """The serving workload: 50,000 requests replayed first all at t = 0
    (the saturated request rate), then as Poisson streams at each of `loads`
    x that rate.  The headline figures are those at `headline_load`."""
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

    def ring():
        return serve.HostRing(ring_t.data_ptr(), ring_words)

    server = m.MontServer(synth.PRIMES, 21, budget, slots=slots, max_batch_coeffs=batch_coeffs)
    # warm-up: a short closed-loop burst
    warm = make()[:500]
    serve.run_stream(server, warm, np.zeros(len(warm)), ring=ring())
    # saturation: every request arrives at t = 0
    lat_s, st_s, mk_s = serve.run_stream(server, make(), np.zeros(n), ring=ring())
    assert np.all(st_s == 0), "serve: a request failed"
    rate_sat = n / mk_s
    sweep = []
    checked = None
    for load in loads:
        lam = load * rate_sat
        arrivals = synth.poisson_arrivals(n, lam, synth.SEED_SERVE, 2)
        b0 = server.stats()["batches"]
        reqs = make()
        lat, st, mk = serve.run_stream(server, reqs, arrivals, ring=ring())
        assert np.all(st == 0), "serve: a request failed at load %.2f" % load
        if load == headline_load:
            checked = check_served(reqs, lens, primes, pools, off_a, off_b, ring_t, ring_words, load)
        sweep.append({"load": load, "lambda_per_s": lam, "value": coeffs / mk / 1e9, "unit": "Gcoef/s",
                      "requests_per_s": n / mk, "makespan_s": mk, "batches": server.stats()["batches"] - b0,
                      **serve.latency_summary(lat)})
    stats = server.stats()
    server.close()
    head = min(sweep, key=lambda r: abs(r["load"] - headline_load))
    return {"workload": "50,000 requests, L log-uniform in [2^8, 2^20], primes uniform from the three Fourier "
                        "primes, Poisson arrivals; operands from a seeded pinned host pool, results copied back",
            "value": head["value"], "unit": "Gcoef/s", "requests_per_s": head["requests_per_s"],
            "makespan_s": head["makespan_s"], "lambda_per_s": head["lambda_per_s"], "load": head["load"],
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "mean_ms": head["mean_ms"], "max_ms": head["max_ms"],
            "saturated": {"requests_per_s": rate_sat, "Gcoef_s": coeffs / mk_s / 1e9, **serve.latency_summary(lat_s)},
            "load_sweep": sweep, "parity": checked, "budget_bytes": budget, "slots": slots,
            "max_batch_coeffs": batch_coeffs,
            "batches": stats["batches"], "peak_bytes": stats["peak_bytes"],
            "latency": "host clock, arrival (scheduled) to completion reported by mont_server_progress"}
