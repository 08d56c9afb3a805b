#!/usr/bin/env python3
"""Benchmark of the Montgomery multiplication hot path on one GB300 per rank.

Workload (one step): elementwise mont_mul (a b R^-1 mod P) and mont_fma
((a b R^-1 + c) mod P) over 2^28 uint32 residues per operand, uniform in
[0, P), for each of the Fourier primes 2013265921, 469762049 and 754974721:
six kernel launches, 6 x 2^28 modular multiplications.  Each operand is
1 GiB, far larger than L2, so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  `value` is Gmulmod/s over all ranks (weak
scaling: each rank runs its own replica of the workload).  `roofline` is
the dominant kernel's algorithmic bytes per launch over its CUDA-event
duration, against the measured HBM copy bandwidth.  `cpu_baseline` is the
CPU oracle timed on the host cores on one full step of the same workload.

--impl reference times the CPU oracle itself on a bounded sample of the
same workload per step (there is no reference implementation to install:
the paper publishes no code).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1609_00999_gb300 import synth  # noqa: E402

N_ELEM = 1 << 28
OPS = ("mont_mul", "mont_fma")
BYTES_PER_ELEM = {"mont_mul": 12, "mont_fma": 16}
METRIC = "Gmulmod/s (elementwise mont_mul + mont_fma)"
UNIT = "Gmulmod/s"
WORKLOAD = ("elementwise mont_mul + mont_fma over 2^28 uint32 residues per operand, uniform in [0,P), "
            "P in {2013265921, 469762049, 754974721}")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("gb300", "reference"), default="gb300")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--log2n", type=int, default=28, help="elements per operand (default 2^28)")
    ap.add_argument("--batch-config", default=None,
                    help="uneven section: fixed launch shape CTAS_PER_SM,ORDER,KERNEL instead of autotuning")
    ap.add_argument("--sections", default="probe,roundtrip,ntt,uniform,reductions,uneven,serve",
                    help="extra sections to run (comma list of probe, roundtrip, ntt, uniform, reductions, uneven, "
                         "serve; empty for none)")
    ap.add_argument("--no-sections-all-ranks", dest="sections_all_ranks", action="store_false",
                    help="with more than one rank, skip the extra sections (default: every rank runs them)")
    ap.add_argument("--no-per-product", action="store_true",
                    help="skip the one-launch-per-product comparison of the uneven batch")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist=None, device=None):
    """Largest value over all ranks (the contract's timing rule); identity
    without a process group.  Works with nccl (device tensor) and gloo (CPU)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def recorded_traffic(kernel_key, n_elem):
    """DRAM bytes per launch from the committed ncu record (profiles/ncu_traffic.json),
    scaled to n_elem, or None when the kernel's sources changed since the
    counters were taken."""
    import bench_polymul as bp
    return bp.recorded_traffic(kernel_key, n_elem)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if self.bus_id:
            mine = [r for r in rows if r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if rows:
            idx = rows[0][0]
            rows = [r for r in rows if r[0] == idx]
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[6:10]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def host_link(torch, h_in, d_in, h_out, d_out, reps=3):
    """Copy-engine rates between pinned host memory and the device (GB/s):
    one stream each way alone, then both at once, timed with CUDA events."""
    nbytes = h_in.numel() * h_in.element_size()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def rate(fn, total):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return total * reps / (e0.elapsed_time(e1) / 1e3) / 1e9

    def h2d():
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        torch.cuda.current_stream().wait_stream(s1)

    def d2h():
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)
        torch.cuda.current_stream().wait_stream(s2)

    def both():
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)
        torch.cuda.current_stream().wait_stream(s1)
        torch.cuda.current_stream().wait_stream(s2)

    return {"h2d_gbs": rate(h2d, nbytes), "d2h_gbs": rate(d2h, nbytes), "both_total_gbs": rate(both, 2 * nbytes),
            "bytes_per_copy": nbytes,
            "method": "cudaMemcpyAsync (torch copy_) of a pinned host buffer, CUDA events"}


def run_section(extra, errors, key, fn):
    """Runs one secondary section into extra[key].  A failure (a parity spot
    check, a device error) is recorded in errors[key] and its traceback
    printed to stderr, so the headline measurement is still reported."""
    try:
        extra[key] = fn()
    except Exception as e:  # noqa: BLE001 -- any failure of a section is reported, not raised
        import traceback
        traceback.print_exc(file=sys.stderr)
        errors[key] = "%s: %s" % (type(e).__name__, str(e)[:300])
        try:
            import torch
            if torch.cuda.is_available():
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
        except Exception:  # noqa: BLE001 -- a broken context shows in the next section's error
            pass


def cpu_oracle_step(arrays, n_sample):
    """Oracle mont_mul + mont_fma over the first n_sample elements of each prime's operands."""
    import oracle
    t0 = time.perf_counter()
    for p, (a, b, c) in arrays:
        oracle.mont_mul(p, a[:n_sample], b[:n_sample])
        oracle.mont_fma(p, a[:n_sample], b[:n_sample], c[:n_sample])
    return time.perf_counter() - t0


def run_reference(args, ws, rank):
    """CPU oracle on a bounded sample of the same workload, per step."""
    if rank != 0:
        return
    import oracle
    n_sample = 1 << min(22, args.log2n)
    arrays = []
    for i in range(3):
        p, ops = synth.elementwise_large(i, n=n_sample)
        arrays.append((p, ops))
    for _ in range(args.warmup):
        cpu_oracle_step(arrays, n_sample)
    t = 0.0
    for _ in range(args.steps):
        t += cpu_oracle_step(arrays, n_sample)
    mulmods = args.steps * 3 * 2 * n_sample
    value = mulmods / t / 1e9
    sample = "first 2^%d residues of each operand, 3 primes x {mont_mul, mont_fma}, per step" % (
        n_sample.bit_length() - 1)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded PCG64)",
            "config": {"workload": WORKLOAD, "n_per_operand": 1 << args.log2n,
                       "sample_per_step": n_sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, ws, rank, local):
    import torch
    import paper_1609_00999_gb300 as m
    from paper_1609_00999_gb300 import build as gbuild

    gbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    n = 1 << args.log2n
    arrays, dev = [], []
    for i in range(3):
        p, (a, b, c) = synth.elementwise_large(i, n=n)
        arrays.append((p, (a, b, c)))
        ctx = m.mont_setup(p)
        tens = [torch.from_numpy(x.view(np.int32)).cuda() for x in (a, b, c)]
        dev.append((ctx, tens, torch.empty_like(tens[0])))
    stream = torch.cuda.current_stream()

    def step(events=None):
        for ctx, (a, b, c), out in dev:
            for op in OPS:
                if events is not None:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                if op == "mont_mul":
                    m.mont_mul(ctx, a, b, out=out)
                else:
                    m.mont_fma(ctx, a, b, c, out=out)
                if events is not None:
                    e1 = torch.cuda.Event(enable_timing=True)
                    e1.record(stream)
                    events[op].append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus)
    sampler.start()
    time.sleep(0.3)
    events = {op: [] for op in OPS}
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(events)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    elapsed_ms = max_over_ranks(t0.elapsed_time(t1), dist, "cuda")
    launches = args.steps * len(dev) * len(OPS)
    per_op_ms = {op: [e0.elapsed_time(e1) for e0, e1 in events[op]] for op in OPS}
    mulmods = args.steps * len(dev) * len(OPS) * n * ws
    value = mulmods / (elapsed_ms / 1e3) / 1e9

    dominant = max(OPS, key=lambda op: sum(per_op_ms[op]))
    avg_ms = sum(per_op_ms[dominant]) / len(per_op_ms[dominant])
    alg_bytes = BYTES_PER_ELEM[dominant] * n
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    kernel_key = "k_elementwise<%s>" % ("OP_FMA" if dominant == "mont_fma" else "OP_MUL")
    roofline = {"bound": "hbm", "kernel": kernel_key, "achieved": achieved, "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(kernel_key, n), "algorithmic_bytes": alg_bytes,
                "avg_launch_ms": avg_ms,
                "per_op_avg_ms": {op: sum(v) / len(v) for op, v in per_op_ms.items()},
                "per_op_gbs": {op: BYTES_PER_ELEM[op] * n / (sum(v) / len(v) / 1e3) / 1e9
                               for op, v in per_op_ms.items()}}

    # End to end: the same C-ABI calls on PINNED HOST buffers.  On GB300 the
    # kernels read the operands from host memory and write the results back
    # to host memory over NVLink-C2C in the same pass (no staging copies), so
    # every step moves each mont_mul's 8 B/element in and 4 B out, and each
    # mont_fma's 12 B in and 4 B out, across the link.
    e2e = None
    if args.e2e_steps > 0:
        host = []
        for p, (a, b, c) in arrays:
            hin = [torch.from_numpy(x.view(np.int32)).pin_memory() for x in (a, b, c)]
            hout = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in OPS]
            host.append((hin, hout))

        def e2e_step():
            for (ctx, _, _), (hin, hout) in zip(dev, host):
                m.mont_mul(ctx, hin[0], hin[1], out=hout[0])
                m.mont_fma(ctx, hin[0], hin[1], hin[2], out=hout[1])

        e2e_step()
        torch.cuda.synchronize()
        for (p, (a, b, c)), (hin, hout) in zip(arrays, host):   # result check on a sample
            k = 4096
            import oracle
            assert np.array_equal(hout[0][:k].numpy().view(np.uint32), oracle.mont_mul(p, a[:k], b[:k]))
            assert np.array_equal(hout[1][:k].numpy().view(np.uint32), oracle.mont_fma(p, a[:k], b[:k], c[:k]))
        barrier()
        w0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - w0, dist, "cuda")
        h2d_bytes, d2h_bytes = len(dev) * (8 + 12) * n, len(dev) * (4 + 4) * n
        e2e = {"value": args.e2e_steps * len(dev) * len(OPS) * n * ws / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
               "steps": args.e2e_steps,
               "path": "C-ABI mont_mul/mont_fma on pinned host buffers: kernels read operands from and write "
                       "results to host memory over NVLink-C2C, one stream, no staging copies"}
        link = host_link(torch, host[0][0][0], dev[0][1][0], host[0][1][0], dev[0][2])
        # Ceiling of the step: its host reads at the measured host-to-device
        # rate (the writes, at the device-to-host rate, run beside them).
        t_min = max(h2d_bytes / (link["h2d_gbs"] * 1e9), d2h_bytes / (link["d2h_gbs"] * 1e9))
        link["step_ceiling"] = len(dev) * len(OPS) * n / t_min / 1e9
        link["frac_of_ceiling"] = e2e["value"] / ws / link["step_ceiling"]
        e2e["host_link"] = link
        del host

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        t = cpu_oracle_step(arrays, n)
        cpu = {"value": 3 * 2 * n / t / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "one full step: 2^%d residues x 3 primes x {mont_mul, mont_fma}" % args.log2n}
        n1 = min(n, 1 << 22)
        with oracle.threads(1):
            t1 = cpu_oracle_step(arrays, n1)
        cpu["single_thread"] = {"value": 3 * 2 * n1 / t1 / 1e9, "unit": UNIT, "cores": 1,
                                "sample": "first 2^%d residues of each operand, 3 primes x {mont_mul, mont_fma}"
                                          % (n1.bit_length() - 1)}

    extra, errors = {}, {}
    if ws == 1 or args.sections_all_ranks:
        # Each rank runs the sections on its own replica; rank 0 reports its own.
        import bench_polymul as bp
        peaks = {"hbm_gbs": measured_peaks()[0], "sm_max_mhz": measured_sm_max_mhz(),
                 "sms": torch.cuda.get_device_properties(local).multi_processor_count}
        secs = [x for x in args.sections.split(",") if x]
        sampler2 = ClockSampler(bus)
        sampler2.start()
        cpu_on = not args.no_cpu_baseline and ws == 1 and rank == 0
        cfg = tuple(int(x) for x in args.batch_config.split(",")) if args.batch_config else None

        def probes():
            res = bp.int_probes(m, torch)
            peaks["probe_rates"] = {k: v["ops_per_s"] for k, v in res["kinds"].items()}
            return res

        sections = [
            ("probe", "int_probe", probes),
            ("roundtrip", "roundtrip_65536", lambda: bp.roundtrip_small(m, torch)),
            ("ntt", "ntt_fwd_inv", lambda: bp.ntt_transforms(m, torch, peaks)),
            ("uniform", "polymul_uniform_4096x2048", lambda: bp.uniform_batch(m, torch, peaks, cpu=cpu_on)),
            ("reductions", "reductions_elementwise_2e28", lambda: bp.reductions_elementwise(m, torch, peaks)),
            ("reductions", "polymul_alg2_vs_alg3_4096x2048", lambda: bp.reduction_ab(m, torch)),
            ("uneven", "polymul_uneven_10000",
             lambda: bp.uneven_batch(m, torch, peaks, cpu=cpu_on, per_product=not args.no_per_product, config=cfg)),
            ("serve", "serve_50000", lambda: bp.serve_stream(m, torch)),
        ]
        for name, key, fn in sections:
            if name in secs:
                run_section(extra, errors, key, fn)
        clk = sampler2.stop()
        if secs:
            extra["clocks_polymul_sections"] = clk
        if "int_probe" in extra:
            mhz = (clk or {}).get("sm_mhz") or peaks["sm_max_mhz"]
            bp.probe_per_sm_clock(extra["int_probe"], mhz, peaks["sms"])
        if ws > 1:
            extra["sections_scope"] = "rank 0's replica (every rank ran the same sections on its own GPU)"

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded PCG64)",
                "config": {"workload": WORKLOAD, "n_per_operand": n, "primes": list(synth.PRIMES),
                           "launches_per_step": len(dev) * len(OPS),
                           "l2": "operands (1 GiB each) larger than L2; no flush",
                           "parallelism": "replica per GPU" if ws > 1 else "single GPU"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "cpu_baseline": cpu}
        line.update(extra)
        if errors:
            line["section_errors"] = errors
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    main()
