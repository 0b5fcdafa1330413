"""The span rule of the subsequence FP64 re-scoring, checked on the CPU.

Before re-scoring an end column b in FP64, the GPU (subseq_rescore_kernel in
paper_1811_11076_gb300/csrc/subseq.cu) bounds how far left a match ending at
b can start: a path from start column a to b crosses every column in between,
so its value is at least the sum (DTW) or the maximum (DK) over those columns
of the column's least cell cost.  Walking back from b, it stops at the first
column jj where that sum (DTW) or that column's least cost alone (DK) exceeds
T, a value above the optimum, and re-scores only columns jj + 1 .. b.

Here the optimum for an end b is found by brute force (the whole-match
recursion of Section 2.1, unbanded, against every T[a..b], FP64 oracle) and
its best start must lie inside the span the rule keeps, for T anywhere from
the optimum itself up to the re-scoring margin used on the GPU.
"""
import numpy as np
import pytest

import oracle


def span_start(s, t, b, T, kind):
    """First column the rule keeps for end b and value limit T."""
    acc = 0.0
    for jj in range(b, -1, -1):
        cm = float(np.min(np.sum((s - t[jj]) ** 2, axis=1)))
        if kind == 0:
            acc += cm
            if acc > T:
                return jj + 1
        elif cm > T:
            return jj + 1
    return 0


@pytest.mark.parametrize("kind", [0, 1])
def test_best_start_lies_inside_the_span(kind):
    rng = np.random.default_rng(31 + kind)
    checked = 0
    for _ in range(10):
        d = int(rng.integers(1, 4))
        m = int(rng.integers(3, 7))
        n = int(rng.integers(12, 26))
        s = np.cumsum(rng.standard_normal((m, d)), 0)
        t = np.cumsum(rng.standard_normal((n, d)), 0)
        v, b = oracle.sub_distance(kind, s, t)
        # brute force: the best start of a match ending at b
        best, a_star = np.inf, -1
        for a in range(b + 1):
            seg = t[a:b + 1]
            r = max(m, len(seg))
            val = oracle.dtw(s, seg, r) if kind == 0 else oracle.dk(s, seg, r)
            if val < best:
                best, a_star = val, a
        assert best == pytest.approx(v, rel=1e-12, abs=1e-12)
        # the rule works in DTW units (sum of squared costs) or DK^2
        opt = best if kind == 0 else best * best
        for T in (opt, opt * (1 + 1e-3)):
            a0 = span_start(s, t, b, T, kind)
            assert a0 <= a_star, (kind, m, n, b, a0, a_star)
        checked += 1
    assert checked == 10
