"""GPU parity of the uneven persistent batch (one launch, mixed sizes and
primes) with the CPU oracle, plus graph replay, autotuning, alone-vs-mix
equality and the bounded-wait failure path.  All comparisons bit-exact."""
import numpy as np
import pytest

import oracle
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


def run_packed(m, wl, graph=False, tune=False):
    import torch
    da, db = to_dev(wl.a), to_dev(wl.b)
    dc = torch.full((max(1, wl.c_size),), -1, dtype=torch.int32, device="cuda")
    plan = m.PolymulBatchPlan.from_packed(wl.primes, da, wl.a_off, wl.la, db, wl.b_off, wl.lb, dc, wl.c_off)
    if tune:
        plan.tune(trials=1)
    (plan.run_graph if graph else plan.run)()
    assert plan.status() == m.MONT_OK
    return plan, da, db, dc


def oracle_packed(wl):
    return oracle.polymul_batch(wl.primes, wl.a, wl.a_off, wl.la, wl.b, wl.b_off, wl.lb, wl.c_off, wl.c_size,
                                use_ntt=True)


def mixed_batch(seed=600):
    rng = np.random.default_rng(seed)
    lens = []
    for k in range(0, 22):                      # every power-of-two size 2^0 .. 2^21 at least once
        lo, hi = max(1, (1 << k) // 4), max(1, (1 << k) // 2)
        lens += [(int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1)))]
    lens += [(1, 1), (1, 5000), (3000, 1), (2048, 2048), (2049, 2048), (4096, 4097), (300, 17)]
    lens += [(int(x), int(x)) for x in synth.loguniform_lengths(200, 1 << 4, 1 << 13, seed, 1)]
    primes = synth.choose_primes(len(lens), seed, 2)
    la = [x for x, _ in lens]
    lb = [y for _, y in lens]
    return synth.UnevenBatch(primes, la, lb, (seed,))


def test_mixed_batch_matches_oracle(m):
    wl = mixed_batch()
    plan, _, _, dc = run_packed(m, wl)
    assert np.array_equal(to_host(dc)[:wl.c_size], oracle_packed(wl))


def test_graph_replay_and_tuning_give_identical_results(m):
    wl = mixed_batch(601)
    ref = oracle_packed(wl)
    plan, da, db, dc = run_packed(m, wl, graph=True)
    assert np.array_equal(to_host(dc)[:wl.c_size], ref)
    dc.fill_(-1)
    plan.run_graph()                              # replay: counters are reset by the graph itself
    assert plan.status() == m.MONT_OK
    assert np.array_equal(to_host(dc)[:wl.c_size], ref)
    cfg = plan.tune(trials=1)
    assert cfg.order in (0, 1, 2, 3) and cfg.kernel in (0, 1, 2) and cfg.full_transforms == 0
    assert cfg.ctas_per_sm >= 1 or cfg.kernel == 2
    for order, kernel in ((0, 0), (1, 1), (2, 0), (3, 1), (0, 2)):
        c = m.PolymulBatchConfig(1 + kernel, order, kernel)
        plan.config = c
        dc.fill_(-1)
        plan.run_graph()
        assert plan.status() == m.MONT_OK
        assert np.array_equal(to_host(dc)[:wl.c_size], ref)


def test_job_kind_boundaries(m):
    """Shapes at the edges of each job kind: single-CTA products up to 2^13,
    whole-product jobs for 2^14 and 2^15 (column levels computed while the
    rows are staged, one operand possibly of length 1), column / row /
    column jobs from 2^16 on; exact powers of two and lengths one past."""
    shapes = [(4096, 4097), (8192, 1), (1, 8192), (8193, 1), (1, 12000), (16384, 1), (9000, 7385),
              (1, 32768), (20000, 12769), (16385, 16384), (32768, 32769), (1, 40000), (40000, 3),
              (65536, 65537), (70000, 1)]
    primes = [synth.PRIMES[i % 3] for i in range(len(shapes))]
    wl = synth.UnevenBatch(primes, [x for x, _ in shapes], [y for _, y in shapes], (604,))
    for cfg in (None, (1, 0, 0), (3, 2, 1), (0, 0, 2)):
        import torch
        da, db = to_dev(wl.a), to_dev(wl.b)
        dc = torch.full((wl.c_size,), -1, dtype=torch.int32, device="cuda")
        plan = m.PolymulBatchPlan.from_packed(wl.primes, da, wl.a_off, wl.la, db, wl.b_off, wl.lb, dc, wl.c_off)
        if cfg is not None:
            plan.config = m.PolymulBatchConfig(*cfg)
        plan.run()
        assert plan.status() == m.MONT_OK
        assert np.array_equal(to_host(dc)[:wl.c_size], oracle_packed(wl)), cfg


# Products of N = 2^15 .. 2^17 on both sides of every row boundary of the
# truncated transforms (rows of 2^13 computed = ceil(lc / 2^13)): one row
# fewer than the full transform, the last rows count that still saves a
# row, exact multiples of 2^13, one past them, and asymmetric operands.
TFT_SHAPES = [(16385, 1), (12289, 12288), (12289, 12289), (8192, 8193), (16385, 16385), (24576, 24577),
              (28672, 28673), (28673, 28673), (1, 40960), (40961, 1), (32769, 32769), (40000, 40000),
              (50000, 50000), (61440, 61441), (61441, 61441), (1, 65537), (70000, 1), (100000, 3)]


@pytest.mark.parametrize("full", [0, 1])
def test_truncated_transform_boundaries(m, full):
    """Split products with and without row-granular truncated transforms
    (polymul_batch_config.full_transforms), every launch shape family,
    against the oracle; the descriptors show which products ran truncated."""
    import torch
    primes = [synth.PRIMES[i % 3] for i in range(len(TFT_SHAPES))]
    wl = synth.UnevenBatch(primes, [x for x, _ in TFT_SHAPES], [y for _, y in TFT_SHAPES], (605,))
    ref = oracle_packed(wl)
    da, db = to_dev(wl.a), to_dev(wl.b)
    descs = [m.PolymulDesc(da.data_ptr() + 4 * int(wl.a_off[i]), db.data_ptr() + 4 * int(wl.b_off[i]),
                           0x10 + 4 * int(wl.c_off[i]), int(wl.la[i]), int(wl.lb[i]), int(wl.primes[i]), 0)
             for i in range(len(wl))]
    _, prods = m.polymul_batch_describe(descs, 0, full)
    assert int(prods[:, 3].sum()) == (0 if full else 14)
    for cfg in ((0, 0, 1), (1, 0, 0), (3, 2, 1), (2, 3, 0), (0, 0, 2)):
        dc = torch.full((wl.c_size,), -1, dtype=torch.int32, device="cuda")
        plan = m.PolymulBatchPlan.from_packed(wl.primes, da, wl.a_off, wl.la, db, wl.b_off, wl.lb, dc, wl.c_off)
        plan.config = m.PolymulBatchConfig(cfg[0], cfg[1], cfg[2], full)
        plan.run_graph()
        assert plan.status() == m.MONT_OK
        check_all_products(wl, to_host(dc), ref)


def test_truncated_equals_full_in_the_mix(m):
    """The same mixed batch (every size 2^0 .. 2^21) with truncated
    transforms and with full ones, by the persistent kernel and by the
    phased form (one kernel per job kind, column tiles up to K1 = 8):
    identical results, equal to the oracle."""
    wl = mixed_batch(606)
    ref = oracle_packed(wl)
    plan, _, _, dc = run_packed(m, wl)
    assert plan.config.full_transforms == 0
    assert np.array_equal(to_host(dc)[:wl.c_size], ref)
    for kernel, full in ((0, 1), (2, 0), (2, 1)):
        plan.config = m.PolymulBatchConfig(2, 0, kernel, full)
        dc.fill_(-1)
        plan.run()
        assert plan.status() == m.MONT_OK
        assert np.array_equal(to_host(dc)[:wl.c_size], ref), (kernel, full)
    dc.fill_(-1)
    plan.run_graph()                                    # the phased form captured in a graph
    assert plan.status() == m.MONT_OK
    assert np.array_equal(to_host(dc)[:wl.c_size], ref)


def test_alone_equals_in_the_mix(m):
    """Every product of a mixed batch equals the same product computed alone."""
    wl = mixed_batch(602)
    _, da, db, dc = run_packed(m, wl)
    got = to_host(dc)
    for i in range(len(wl)):
        ao, la = int(wl.a_off[i]), int(wl.la[i])
        bo, lb = int(wl.b_off[i]), int(wl.lb[i])
        co = int(wl.c_off[i])
        alone = to_host(m.polymul(int(wl.primes[i]), da[ao:ao + la], db[bo:bo + lb]))
        assert np.array_equal(got[co:co + la + lb - 1], alone), i


def one_shot(m, wl, ws=None):
    import torch
    da, db = to_dev(wl.a), to_dev(wl.b)
    dc = torch.full((max(1, wl.c_size),), -1, dtype=torch.int32, device="cuda")
    descs = [m.PolymulDesc(da.data_ptr() + 4 * int(wl.a_off[i]), db.data_ptr() + 4 * int(wl.b_off[i]),
                           dc.data_ptr() + 4 * int(wl.c_off[i]), int(wl.la[i]), int(wl.lb[i]), int(wl.primes[i]), 0)
             for i in range(len(wl))]
    need = m.polymul_batch_workspace_bytes(descs)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(1, need), dtype=torch.uint8, device="cuda")
    m.polymul_batch(descs, ws)
    assert m.polymul_batch_check(ws) == m.MONT_OK
    return to_host(dc)[:wl.c_size], ws


def test_one_shot_batch_matches_oracle(m):
    """polymul_batch (no plan, tables in the caller's workspace) on every
    size 2^0 .. 2^21, then a second batch reusing the same workspace."""
    wl = mixed_batch()
    got, ws = one_shot(m, wl)
    assert np.array_equal(got, oracle_packed(wl))
    wl2 = synth.batch_uneven(count=300, hi=1 << 15)
    got2, _ = one_shot(m, wl2, ws)
    assert np.array_equal(got2, oracle_packed(wl2))


def check_all_products(wl, got, ref=None):
    """Every output word of every product equals the oracle's product (all
    of them, in one OpenMP call of the oracle's radix-2 NTT products)."""
    if ref is None:
        ref = oracle_packed(wl)
    bad = np.flatnonzero(got[:wl.c_size] != ref)
    if bad.size:
        first = int(np.searchsorted(wl.c_off.astype(np.int64), bad[0], side="right") - 1)
        raise AssertionError("%d wrong words; first in product %d" % (bad.size, first))


def test_uneven_full_size_exhaustive(m):
    """The whole 10,000-product uneven workload (L log-uniform in [2^6, 2^16],
    primes uniform from the three Fourier primes), tuned and replayed from a
    CUDA graph as the benchmark runs it, twice over the same buffers (which
    start at 0xFFFFFFFF): every output word of every product against the
    oracle."""
    wl = synth.batch_uneven()
    ref = oracle_packed(wl)
    plan, _, _, dc = run_packed(m, wl, graph=True, tune=True)
    check_all_products(wl, to_host(dc), ref)
    dc.fill_(-1)
    plan.run_graph()
    assert plan.status() == m.MONT_OK
    check_all_products(wl, to_host(dc), ref)
    # the same launch shape with every product padded to its full transform,
    # and both transform forms by the other kernel form
    c = plan.config
    assert c.full_transforms == 0
    other = 0 if c.kernel == 2 else 2
    for kernel, full in ((c.kernel, 1), (other, 0), (other, 1)):
        plan.config = m.PolymulBatchConfig(c.ctas_per_sm if kernel != 2 else 0, c.order, kernel, full)
        dc.fill_(-1)
        plan.run_graph()
        assert plan.status() == m.MONT_OK
        check_all_products(wl, to_host(dc), ref)


def test_uneven_config_sample(m):
    """A 600-product slice of the 10,000-product uneven workload (L log-uniform in [2^6, 2^16])."""
    wl_full = synth.batch_uneven(count=600)
    plan, _, _, dc = run_packed(m, wl_full, tune=True)
    assert np.array_equal(to_host(dc)[:wl_full.c_size], oracle_packed(wl_full))


def test_bounded_wait_reports_timeout_and_context_survives(m):
    import torch
    wl = synth.UnevenBatch([synth.P1, synth.P2], [20000, 10], [20000, 10], (603,))   # N = 2^16: cross-CTA waits
    da, db = to_dev(wl.a), to_dev(wl.b)
    dc = torch.zeros(wl.c_size, dtype=torch.int32, device="cuda")
    plan = m.PolymulBatchPlan.from_packed(wl.primes, da, wl.a_off, wl.la, db, wl.b_off, wl.lb, dc, wl.c_off)
    plan.set_wait_limit(20000, 20_000_000)        # 20 ms per wait
    plan.inject_stall()                           # rows wait for a column tile that never finishes
    plan.run()
    assert plan.status() == m.MONT_ETIMEOUT
    # the context is still usable: a fresh plan of the same batch is exact
    _, _, _, dc2 = run_packed(m, wl)
    assert np.array_equal(to_host(dc2)[:wl.c_size], oracle_packed(wl))


def test_batch_argument_errors(m):
    import torch
    d = to_dev(np.ones(8, dtype=np.uint32))
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    bad = [m.PolymulDesc(d.data_ptr(), d.data_ptr(), out.data_ptr(), 0, 4, synth.P1, 0)]
    with pytest.raises(m.MontError) as e:
        m.PolymulBatchPlan(bad)
    assert e.value.code == m.MONT_EINVAL
    huge = [m.PolymulDesc(d.data_ptr(), d.data_ptr(), out.data_ptr(), 1 << 21, 1 << 21, synth.P1, 0)]
    with pytest.raises(m.MontError) as e:
        m.PolymulBatchPlan(huge)
    assert e.value.code in (m.MONT_EUNSUPPORTED, m.MONT_ERANGE)
    empty = m.PolymulBatchPlan([])
    empty.run()
    assert empty.status() == m.MONT_OK
