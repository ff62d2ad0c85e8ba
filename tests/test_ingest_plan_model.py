"""CPU model of the ingest's bucket plan (the kernel that cuts the
histogram of entries over vertex ranges into buckets of consecutive
owners): for skewed, empty, tiny and maximal inputs the buckets cover the
vertices exactly once, in order, their entry bases are the exclusive
prefix of their entries, and their number never exceeds the capacity of
the scatter's shared-memory table.  No GPU involved."""
import re
import os

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2103_00154_gb300", "csrc",
                   "ingest.cu")


def _const(name):
    text = open(SRC).read()
    m = re.search(rf"constexpr \w+ {name} = ([^;]+);", text)
    expr = m.group(1)
    for other in re.findall(r"k[A-Z]\w+", expr):
        expr = expr.replace(other, str(_const(other)))
    return int(eval(expr.replace("ull", "").replace("u", "")))


K_RANGES = _const("kRangesMax")
K_TARGET = _const("kBucketTarget")
K_MIN = _const("kBucketMinEntries")
K_SPAN = _const("kSpanMax")
K_SPAN_CUTS = _const("kSpanCutBuckets")
K_BUCKETS = _const("kBucketsMax")


def plan_for(n):
    rshift = 0
    while (n + (1 << rshift) - 1) >> rshift > K_RANGES:
        rshift += 1
    nranges = (n + (1 << rshift) - 1) >> rshift
    width = 1 << rshift
    cut = K_SPAN // width if width <= K_SPAN else 1
    need = (nranges + K_SPAN_CUTS - 1) // K_SPAN_CUTS
    return rshift, nranges, max(cut, need)


def plan(n, range_cnt):
    rshift, nranges, span_cut = plan_for(n)
    assert len(range_cnt) == nranges
    total = int(np.sum(range_cnt))
    target = max((total + K_TARGET - 1) // K_TARGET, K_MIN)
    pre = np.concatenate([[0], np.cumsum(range_cnt, dtype=np.int64)])
    v0, base, bucket_of = [], [], np.empty(nranges, np.int64)
    for r in range(nranges):
        prev = 0 if r == 0 else pre[r - 1]
        if r == 0 or pre[r] // target != prev // target or r % span_cut == 0:
            v0.append(r << rshift)
            base.append(int(pre[r]))
        bucket_of[r] = len(v0) - 1
    v0.append(n)
    base.append(total)
    return rshift, span_cut, np.array(v0, np.int64), np.array(base, np.int64), bucket_of


def _check(n, range_cnt):
    rshift, span_cut, v0, base, bucket_of = plan(n, range_cnt)
    F = len(v0) - 1
    assert F <= K_BUCKETS
    assert F < 65536  # bucket ids are kept as 16-bit numbers
    assert v0[0] == 0 and v0[-1] == n and np.all(np.diff(v0) > 0)
    # each bucket's entries are those of its ranges
    sums = np.bincount(bucket_of, weights=range_cnt, minlength=F).astype(np.int64)
    np.testing.assert_array_equal(np.diff(base), sums)
    # every range lies inside its bucket's vertex span
    r = np.arange(len(range_cnt))
    assert np.all(v0[bucket_of] <= (r << rshift)) and np.all((r << rshift) < v0[bucket_of + 1])
    assert np.all(v0[:-1] < (1 << 31))


@pytest.mark.parametrize("n", [1, 2, 31, 1000, 65536, 65537, 1 << 20, (1 << 24) + 3, 1 << 27, (1 << 31) - 1])
def test_plan_covers_vertices_with_bounded_bucket_count(n):
    rng = np.random.default_rng(n % 1000)
    _, nranges, _ = plan_for(n)
    if nranges > 70000:
        pytest.fail("more ranges than the histogram holds")
    for kind in ("uniform", "power", "one_hub", "empty", "every_other"):
        if kind == "uniform":
            c = rng.integers(0, 64, nranges)
        elif kind == "power":
            c = (1e6 / (np.arange(nranges) + 1) ** 1.1).astype(np.int64)
        elif kind == "one_hub":
            c = np.zeros(nranges, np.int64)
            c[nranges // 2] = 2 ** 33 - 2
        elif kind == "empty":
            c = np.zeros(nranges, np.int64)
        else:
            c = np.where(np.arange(nranges) % 2 == 0, 1 << 20, 0)
        _check(n, np.asarray(c, np.int64))
