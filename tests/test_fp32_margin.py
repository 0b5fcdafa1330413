"""The FP32 error bound behind the scan's exactness margins, checked on the CPU.

The scan computes DTW and DK in FP32 and re-scores in FP64 every result within
relative w of the k-th one (w = 2 (max_path + d + 8) u for DTW, 2 (d + 8) u for
DK, u = 2^-24; margins_for in paper_1811_11076_gb300/csrc/api.cu).  That is
exact if one FP32 value is within w / 2 of its FP64 value.  This evaluates the
banded recursions (Section 2.1) in FP32 scalar arithmetic, with each point cost
a chain of fused multiply-adds as in the kernels, on series far from the
origin and on near-duplicates (tiny costs, long paths), and checks the relative
error against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle

U = 2.0 ** -24


def fma32(a, b, c):
    return np.float32(float(a) * float(b) + float(c))


def dp32(s, t, r, kind):
    m, n = len(s), len(t)
    inf = np.float32(np.inf)
    D = np.full((m + 1, n + 1), inf, dtype=np.float32)
    D[0, 0] = 0.0
    for i in range(1, m + 1):
        for j in range(max(1, i - r), min(n, i + r) + 1):
            c = np.float32(0.0)
            for k in range(s.shape[1]):
                e = np.float32(s[i - 1, k] - t[j - 1, k])
                c = fma32(e, e, c)
            best = min(D[i - 1, j], D[i, j - 1], D[i - 1, j - 1])
            D[i, j] = np.float32(c + best) if kind == 0 else max(c, best)
    return float(D[m, n])


@pytest.mark.parametrize("kind", [0, 1])
def test_fp32_value_within_half_the_margin(kind):
    rng = np.random.default_rng(7 + kind)
    worst = 0.0
    for trial in range(12):
        d = int(rng.integers(1, 9))
        m = int(rng.integers(20, 48))
        n = m + int(rng.integers(-3, 4))
        r = max(abs(m - n), int(rng.integers(2, 10)))
        base = np.cumsum(rng.standard_normal((max(m, n), d)), 0) + rng.choice([0.0, 500.0])
        s = base[:m].astype(np.float32)
        if trial % 2:
            t = (base[:n] + 1e-3 * rng.standard_normal((n, d))).astype(np.float32)
        else:
            t = (np.cumsum(rng.standard_normal((n, d)), 0) + base[0]).astype(np.float32)
        v32 = dp32(s, t, r, kind)
        v64 = oracle.dtw(s.astype(np.float64), t.astype(np.float64), r) if kind == 0 else \
            oracle.dk(s.astype(np.float64), t.astype(np.float64), r) ** 2
        if not np.isfinite(v64) or v64 == 0.0:
            continue
        w = 2 * (m + n + d + 8) * U if kind == 0 else 2 * (d + 8) * U
        err = abs(v32 - v64) / v64
        worst = max(worst, err / (w / 2))
        assert err <= w / 2, (trial, kind, err, w)
    assert worst > 0.0
