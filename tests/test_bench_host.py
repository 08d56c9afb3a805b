"""Host-side checks of the bench's work accounting (no GPU).

The roofline figures divide algorithmic work by kernel time, so the counts
must describe the transform the kernels run: levels 0 .. K-1 of a
Cooley-Tukey forward transform over 2^l blocks of size N / 2^l, block i
multiplying by w^(brev_l(i) N / 2^(l+1)), output in bit-reversed order
(Sec. 4: the twiddle multiply is the REDC of Alg. 2).  The brute-force walk
below runs that transform, checks it against the DFT, and counts its
butterflies by whether the twiddle is 1.
"""
import numpy as np
import pytest

import bench_polymul as bp
import oracle
from paper_1609_00999_gb300 import synth


def _brev(i, bits):
    return int(format(i, f"0{bits}b")[::-1], 2) if bits else 0


def _ct_forward_counting(p, x):
    n = len(x)
    k = n.bit_length() - 1
    w = int(oracle.root_of_unity(p, n))
    a = [int(v) for v in x]
    trivial = nontrivial = 0
    for level in range(k):
        half = n >> (level + 1)
        for blk in range(1 << level):
            tw = pow(w, _brev(blk, level) * half, p)
            base = blk * 2 * half
            for j in range(base, base + half):
                u, v = a[j], a[j + half] * tw % p
                a[j], a[j + half] = (u + v) % p, (u - v) % p
                if tw == 1:
                    trivial += 1
                else:
                    nontrivial += 1
    return a, trivial, nontrivial


@pytest.mark.parametrize("k", range(1, 11))
def test_butterfly_classes_match_op_count(k):
    n = 1 << k
    p = synth.P1
    x = synth.residues(n, p, 4242, k)
    y, trivial, nontrivial = _ct_forward_counting(p, x)
    ref = oracle.dft(p, x)
    assert [y[_brev(i, k)] for i in range(n)] == [int(v) for v in ref]
    assert trivial == n - 1
    assert trivial + nontrivial == (n // 2) * k
    assert bp.int_ops_ntt(n, False) == 10 * nontrivial + 4 * trivial
    assert bp.int_ops_ntt(n, True) == 9 * nontrivial + 4 * trivial + 6 * n
    la, lb = n // 2, n // 2
    assert bp.int_ops_polymul(n, la, lb) == (2 * (10 * nontrivial + 4 * trivial) + 9 * nontrivial + 4 * trivial
                                             + 6 * n + 6 * lb)
    # the operation classes the measured floor weights: level 0 (n/2
    # butterflies, all in block 0, twiddle 1 on reduced inputs), the other
    # twiddle-1 butterflies, and the rest
    fwd = bp.op_counts_ntt(n, False)
    assert fwd == {"ct": nontrivial, "ct_first": n // 2, "ct_one": trivial - n // 2}
    assert bp.op_counts_ntt(n, True) == {"gs": nontrivial, "gs_one": trivial, "redc": n}
    prod = bp.op_counts_polymul(n, lb)
    assert prod == {"ct": 2 * nontrivial, "ct_first": n, "ct_one": 2 * (trivial - n // 2), "gs": nontrivial,
                    "gs_one": trivial, "redc": n + lb}


def test_measured_floor_arithmetic():
    """floor = sum over classes of count / rate; frac = floor / time."""
    counts = bp.add_counts({}, bp.op_counts_polymul(4096, 2048), 4096)
    rates = {k: 1e12 for k in bp.OP_CLASSES}
    floor = bp.floor_seconds(counts, rates)
    assert floor == pytest.approx(sum(counts.values()) / 1e12)
    peaks = {"sm_max_mhz": 2070.0, "sms": 152, "probe_rates": rates}
    r = bp.int_roofline("k_polymul<12, RedAlg2>", 1e9, counts, 2 * floor * 1e3, peaks)
    assert r["frac"] == pytest.approx(0.5) and r["peak_source"].startswith("measured")
    assert r["achieved"] / r["peak"] == pytest.approx(0.5)
    r2 = bp.int_roofline("k_polymul<12, RedAlg2>", 1e9, counts, 1.0, {"sm_max_mhz": 2070.0})
    assert r2["peak_source"].startswith("derived")
    assert bp.op_counts_polymul(1, 1) == {"redc": 2}


def test_batch_hbm_bytes_pass_structure():
    # One pass for products held in one CTA.
    assert bp.batch_hbm_bytes(1 << 13, 4000, 4000) == 4 * (4000 + 4000 + 7999)
    # 2^14 / 2^15: operands re-read once per extra row, product rows out and back.
    io = 4 * (9000 + 8000 + 16999)
    assert bp.batch_hbm_bytes(1 << 15, 9000, 8000) == io + 4 * 3 * 17000 + 8 * (1 << 15)
    # Larger: forward scratch (2N) and product rows (N) each out and back.
    n = 1 << 17
    io = 4 * (70000 + 60000 + 129999)
    assert bp.batch_hbm_bytes(n, 70000, 60000) == io + 4 * 6 * n
    lens = np.array([1 << 12, 1 << 14, 1 << 16])
    sizes = [1 << int(2 * L - 2).bit_length() for L in lens]
    vals = [bp.batch_hbm_bytes(s, int(L), int(L)) for s, L in zip(sizes, lens)]
    assert vals == sorted(vals)


def test_section_failure_is_recorded_not_raised(capsys):
    """A failing secondary section leaves the others and the headline line
    intact and is reported under its key."""
    import bench
    extra, errors = {}, {}
    bench.run_section(extra, errors, "first", lambda: {"value": 1.0})

    def broken():
        raise AssertionError("batch parity spot check failed")

    bench.run_section(extra, errors, "second", broken)
    bench.run_section(extra, errors, "third", lambda: {"value": 3.0})
    assert extra == {"first": {"value": 1.0}, "third": {"value": 3.0}}
    assert errors == {"second": "AssertionError: batch parity spot check failed"}
    assert "batch parity spot check failed" in capsys.readouterr().err


def test_served_results_check_reads_the_ring_as_placed():
    """The bench's oracle check of served results: regions handed out by the
    result ring in request order (with wrap-around), filled with the
    oracle's products; the check passes, and fails on a planted wrong word
    in a request it samples."""
    import torch
    from paper_1609_00999_gb300 import serve
    n, ring_words, pool_n = 60, 4096, 1 << 12
    rng = np.random.default_rng(5)
    lens = rng.integers(8, 200, size=n).astype(np.int64)
    primes = np.asarray([synth.PRIMES[i % 3] for i in range(n)], dtype=np.uint32)
    pools = {p: torch.from_numpy(synth.residues(pool_n, p, 77, i).view(np.int32)) for i, p in enumerate(synth.PRIMES)}
    off_a = rng.integers(0, pool_n - 200, size=n)
    off_b = rng.integers(0, pool_n - 200, size=n)
    ring_t = torch.zeros(ring_words, dtype=torch.int32)
    ring = serve.HostRing(ring_t.data_ptr(), ring_words)
    reqs = serve.make_requests(primes, lens, lens, np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int64))
    view = ring_t.numpy().view(np.uint32)
    for i in range(n):                       # in order, five in flight, so regions advance and wrap around
        lc = int(2 * lens[i] - 1)
        if i >= 5:
            ring.release(i - 5)
        ptr = ring.alloc(i, lc)
        assert ptr is not None
        reqs["c"][i] = ptr
        p = int(primes[i])
        pool = pools[p].numpy().view(np.uint32)
        start = (ptr - ring_t.data_ptr()) // 4
        view[start:start + lc] = oracle.polymul_ntt(p, pool[off_a[i]:off_a[i] + lens[i]],
                                                    pool[off_b[i]:off_b[i] + lens[i]])
    msg = bp.check_served(reqs, lens, primes, pools, off_a, off_b, ring_t, ring_words, 0.8, sample=6)
    assert "intact results" in msg and int(msg.split(" of the ")[1].split()[0]) >= 6
    last = n - 1
    start = (int(reqs["c"][last]) - ring_t.data_ptr()) // 4
    view[start + 3] ^= 1                      # the last request is always checked
    with pytest.raises(AssertionError):
        bp.check_served(reqs, lens, primes, pools, off_a, off_b, ring_t, ring_words, 0.8, sample=6)
