"""Shared-memory bank accounting of the register passes (CPU).

Mirrors the pass geometry of ``csrc/ntt_core.cuh`` (``Sched``, ``SchedFor``,
``PassGeom`` with its group remap for the padded layout) and counts, for
every warp access of every pass, the shared-memory wavefronts on the padded
layout (word j + (j >> 5), 32 banks of 4 bytes): the middle passes of
2^11 .. 2^13 were 2-way conflicted before the remap; with it every pass of
2^11 .. 2^14 (the single-CTA transforms and products, and the rows of the
large transforms and batches) is conflict-free."""
import pytest


def ilog2(x):
    return 0 if x <= 1 else 1 + ilog2(x // 2)


def nt_of(logn):
    return 1 if logn <= 4 else (256 if logn == 13 else (512 if logn == 14 else 1 << (logn - 4)))


def sched(logn, nt):
    emax = 5 if logn - ilog2(nt) >= 5 else 4
    np_ = (logn + emax - 1) // emax
    lv = [logn // np_ + (1 if i < logn % np_ else 0) for i in range(np_)]
    return [(sum(lv[:i]), lv[i]) for i in range(np_)]


def grp(tid, hmin, g, nt, remap):
    d = 32 // g if g < 32 else 1
    if not (remap and 2 <= hmin < 32 and g < 32 and hmin * g >= 32 and nt % (32 * d) == 0):
        return tid
    nb = 32 // hmin
    w, l = divmod(tid, 32)
    block = (w // d) * (d * nb) + (w % d) + (l // hmin) * d
    return block * hmin + l % hmin


def wavefronts(words):
    banks = {}
    for w in set(words):
        banks.setdefault(w % 32, set()).add(w)
    return max(len(v) for v in banks.values())


def pass_worst(logn, nt, remap):
    """Worst wavefronts per warp access, per pass; also checks that every
    element is touched exactly once per pass."""
    out = []
    for s0, e in sched(logn, nt):
        g, log_hmin = 1 << e, logn - s0 - e
        hmin, gpt = 1 << log_hmin, (1 << logn) // (1 << e) // nt
        qs = [grp(t, hmin, g, nt, remap) for t in range(nt)]
        assert sorted(qs) == list(range(nt))
        seen, worst = set(), 1
        for r in range(gpt):
            for w0 in range(0, nt, 32):
                for t in range(g):
                    words = []
                    for tid in range(w0, min(nt, w0 + 32)):
                        q = qs[tid] + nt * r
                        j = ((q >> log_hmin) << (logn - s0)) + (q & (hmin - 1)) + t * hmin
                        seen.add(j)
                        words.append(j + (j >> 5))
                    worst = max(worst, wavefronts(words))
        assert seen == set(range(1 << logn))
        out.append(worst)
    return out


@pytest.mark.parametrize("logn", range(11, 15))
def test_passes_conflict_free_with_remap(logn):
    assert pass_worst(logn, nt_of(logn), True) == [1] * len(sched(logn, nt_of(logn)))


def test_middle_pass_conflicted_without_remap():
    # 4096 points on 256 threads: passes of HMIN 256, 16, 1; the middle one
    # spans two blocks per warp whose banks overlap
    assert pass_worst(12, 256, False) == [1, 2, 1]
    assert pass_worst(13, 256, False) == [1, 2, 1]


@pytest.mark.parametrize("logn", range(5, 11))
def test_small_transforms_bounded(logn):
    # 2^9 and 2^10 keep 4-way conflicts in their middle pass (too few blocks
    # to space a warp's segments apart); nothing is worse
    worst = pass_worst(logn, nt_of(logn), True)
    assert max(worst) <= 4
    assert max(worst) == (4 if logn in (9, 10) else 1)
