"""Host-side job lists of the persistent batch kernel (no GPU needed).

The kernel's progress rests on one property of its job list: every job
waits only on jobs earlier in the list (a row job on all column tiles of
its product, an output-tile job on all rows of its product), so the
earliest unfinished job can always run.  These tests build the job lists
for every job order from the host builder the kernel uses and check that
property, that every product is covered exactly once by jobs of the kind
its size calls for, and the descriptor checks."""
import pytest

from paper_1609_00999_gb300 import build as gbuild
from paper_1609_00999_gb300 import synth

SMALL, COLF, ROW, COLI, WHOLE = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def m():
    gbuild.build()
    import paper_1609_00999_gb300 as m
    return m


def fake_descs(m, la, lb, primes):
    """Descriptors with distinct, non-overlapping addresses that the host
    builder only compares, never dereferences."""
    out, base = [], 1 << 40
    for x, y, p in zip(la, lb, primes):
        a, b, c = base, base + 4 * int(x), base + 4 * (int(x) + int(y))
        base += 4 * (2 * (int(x) + int(y))) + 4096
        out.append(m.PolymulDesc(a, b, c, int(x), int(y), int(p), 0))
    return out


def kernel_order_lc(la, lb):
    """Output lengths in the kernel's product order: products with N <= 2^13
    first, stably sorted by log2 N, then the others in descriptor order."""
    lc = [int(x) + int(y) - 1 for x, y in zip(la, lb)]
    k = [(c - 1).bit_length() for c in lc]
    small = sorted((i for i in range(len(lc)) if k[i] <= 13), key=lambda i: k[i])
    return [lc[i] for i in small] + [lc[i] for i in range(len(lc)) if k[i] > 13]


def check_job_list(jobs, prods, lc=None):
    count = len(prods)
    small = [0] * count
    whole = [0] * count
    colf, row, coli = [0] * count, [0] * count, [0] * count
    for kind, k, prod, idx in jobs.tolist():
        if kind == SMALL:
            assert idx >= 1 and prod + idx <= count
            for q in range(prod, prod + idx):
                assert prods[q][0] == k and k <= 13
                small[q] += 1
        elif kind == WHOLE:
            assert prods[prod][0] == k and 14 <= k <= 15
            whole[prod] += 1
        elif kind == COLF:
            assert prods[prod][0] == k >= 16 and idx < prods[prod][1]
            colf[prod] += 1
        elif kind == ROW:
            assert colf[prod] == prods[prod][1], "row job before all column tiles of its product"
            assert idx < prods[prod][2]
            row[prod] += 1
        elif kind == COLI:
            assert row[prod] == prods[prod][2], "output tile before all rows of its product"
            assert idx < prods[prod][1]
            coli[prod] += 1
        else:
            raise AssertionError("unknown job kind %d" % kind)
    for q in range(count):
        k, ntiles, nrows, tft = (int(v) for v in prods[q])
        if k <= 13:
            assert small[q] == 1 and whole[q] == colf[q] == row[q] == coli[q] == 0, q
            assert tft == 0
        elif k <= 15:
            assert whole[q] == 1 and small[q] == colf[q] == row[q] == coli[q] == 0, q
        else:
            assert (colf[q], row[q], coli[q]) == (ntiles, nrows, ntiles) and small[q] == whole[q] == 0, q
        if k > 13:
            # a truncated product computes just the rows of 2^13 its output
            # reaches; the others compute all 2^(k - 13)
            if tft:
                assert 2 <= k - 13 <= 4 and nrows < 1 << (k - 13)
            else:
                assert nrows == 1 << (k - 13)
    if lc is not None:
        for q in range(count):
            k, _, nrows, tft = (int(v) for v in prods[q])
            if tft:
                assert (nrows - 1) * 8192 < lc[q] <= nrows * 8192, q


@pytest.mark.parametrize("full", [0, 1])
@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_uneven_workload_job_lists(m, order, full):
    """The 10,000-product uneven workload (sizes and primes only), with
    truncated transforms (full = 0) and without."""
    lens = synth.loguniform_lengths(10000, 1 << 6, 1 << 16, synth.SEED_BATCH_UNEVEN, 0)
    primes = synth.choose_primes(10000, synth.SEED_BATCH_UNEVEN, 1)
    jobs, prods = m.polymul_batch_describe(fake_descs(m, lens, lens, primes), order, full)
    check_job_list(jobs, prods)
    tft = prods[:, 3]
    assert (tft.any() if full == 0 else not tft.any())


def test_tft_rows_follow_the_output_length(m):
    """Products kept in descriptor order among the split ones: rows computed
    = ceil(lc / 2^13) exactly when that leaves rows of the full transform
    unused and 2 <= log2 N - 13 <= 4."""
    la = [16385, 24577, 20000, 40000, 40960, 65536, 32769, 70000, 100000, 131072]
    lb = [1, 1, 4, 1, 1, 1, 1, 60000, 1, 1]
    primes = [synth.PRIMES[i % 3] for i in range(len(la))]
    jobs, prods = m.polymul_batch_describe(fake_descs(m, la, lb, primes), 0, 0)
    lc = [x + y - 1 for x, y in zip(la, lb)]
    check_job_list(jobs, prods, lc)
    got = [(int(p[0]), int(p[2]), int(p[3])) for p in prods]
    want = []
    for c in lc:
        k = (c - 1).bit_length()
        need = -(-c // 8192)
        t = int(2 <= k - 13 <= 4 and need < 1 << (k - 13))
        want.append((k, need if t else 1 << (k - 13), t))
    assert got == want


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_mixed_sizes_job_lists(m, order):
    """Every size 2^0 .. 2^21, asymmetric operands, primes mixed."""
    la, lb = [], []
    for k in range(22):
        n = 1 << k
        la += [max(1, n // 2), 1, max(1, n // 4)]
        lb += [max(1, n // 2), max(1, n - 1), max(1, n // 2 + 1)]
    primes = [synth.PRIMES[i % 3] for i in range(len(la))]
    jobs, prods = m.polymul_batch_describe(fake_descs(m, la, lb, primes), order)
    check_job_list(jobs, prods)
    assert {int(p[0]) for p in prods} >= set(range(0, 22))


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_random_batches_job_lists(m, order):
    """40 seeded random batches of 1 to 300 products, lengths log-uniform in
    [1, 2^20] and drawn separately for a and b: many with only a few split
    products, fewer than the pipelined orders' lag of 32 or 64."""
    import numpy as np
    rng = np.random.default_rng(8800 + order)
    for trial in range(40):
        count = int(rng.integers(1, 301))
        la = np.exp(rng.uniform(0, np.log(1 << 20), count)).astype(np.int64).clip(1, 1 << 20)
        lb = np.exp(rng.uniform(0, np.log(1 << 20), count)).astype(np.int64).clip(1, 1 << 20)
        primes = [synth.PRIMES[i] for i in rng.integers(0, 3, count)]
        d = fake_descs(m, la, lb, primes)
        jobs, prods = m.polymul_batch_describe(d, order)
        check_job_list(jobs, prods, kernel_order_lc(la, lb))


def test_describe_rejects_bad_input(m):
    d = fake_descs(m, [10], [10], [synth.P1])
    with pytest.raises(m.MontError):
        m.polymul_batch_describe(d, 4)                       # no such order
    big = fake_descs(m, [1 << 21], [1 << 21], [synth.P1])    # N = 2^22 > 2^21
    with pytest.raises(m.MontError) as e:
        m.polymul_batch_describe(big, 0)
    assert e.value.code == m.MONT_EUNSUPPORTED
    zero = fake_descs(m, [0], [5], [synth.P1])
    with pytest.raises(m.MontError) as e:
        m.polymul_batch_describe(zero, 0)
    assert e.value.code == m.MONT_EINVAL


def test_one_shot_workspace_layout(m):
    """polymul_batch's workspace: counters (2 + 2 count words), product table
    (64 B per product), the phased form's job lists (16 B per job: the
    column, row and output-tile jobs of every product above 2^13, truncated
    transforms on), each part rounded up to 256 B, then 2N words of scratch
    per product with N > 2^13."""
    def up(x):
        return (x + 255) // 256 * 256

    lens = synth.loguniform_lengths(400, 1 << 4, 1 << 17, 4321, 0)
    primes = synth.choose_primes(400, 4321, 1)
    descs = fake_descs(m, lens, lens, primes)
    jobs, prods = m.polymul_batch_describe(descs, 0)
    njobs = sum(1 for j in jobs.tolist() if j[0] in (COLF, ROW, COLI))
    njobs += sum(2 * int(prods[j[2]][1]) + int(prods[j[2]][2]) for j in jobs.tolist() if j[0] == WHOLE)
    scratch = 0
    for L in lens:
        n = 1 << int(2 * int(L) - 2).bit_length()
        if n > 1 << 13:
            scratch += 2 * n
    want = up(4 * (2 + 2 * len(descs))) + up(64 * len(descs)) + up(16 * njobs) + 4 * scratch
    assert m.polymul_batch_workspace_bytes(descs) == want


def test_bench_row_rule_matches_the_builder(m):
    """The bench's work and byte counts of truncated products use the same
    rows-computed rule as the batch builder (compared on the uneven
    workload's sizes)."""
    import bench_polymul as bp
    lens = synth.loguniform_lengths(10000, 1 << 6, 1 << 16, synth.SEED_BATCH_UNEVEN, 0)
    primes = synth.choose_primes(10000, synth.SEED_BATCH_UNEVEN, 1)
    _, prods = m.polymul_batch_describe(fake_descs(m, lens, lens, primes), 0, 0)
    lc = kernel_order_lc(lens, lens)
    for (k, _, nrows, tft), c in zip(prods.tolist(), lc):
        rows = bp.tft_rows(1 << k, c)
        assert (rows is not None) == bool(tft)
        if tft:
            assert rows == nrows
