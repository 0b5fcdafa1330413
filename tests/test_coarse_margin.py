"""The rounding margin of the coarse LB stage, checked on the CPU (no GPU).

The coarse stage (paper_1811_11076_gb300/csrc/lbcoarse.cu) compares an FP32
segment-box bound with a widened limit
    lim_c = ((sqrt(lim) + c2) / (1 - c1))^2,  c1 = (K/2 + 3) u,
    c2 = sqrt(K W) u M,  u = 2^-24,
(K terms, segment width W, M the largest coordinate magnitude of the
database), so that no pair whose exact coarse bound is within `lim` is pruned.
This emulates the kernel's FP32 arithmetic in numpy (segment means rounded once
to FP32 and scaled by sqrt(W), box bounds scaled likewise, gaps as max(lo - x,
x - hi, 0), one fused multiply-add chain per segment, segments summed in
order) and checks that the FP32 bound never exceeds the limit computed from
the exact FP64 bound, on smooth data far from the origin, where the rounding
of the means (the c2 term) matters most.
"""
import math

import numpy as np
import pytest

U = 2.0 ** -24


def coarse_limit(lim, K, W, M):
    c1 = (0.5 * K + 3.0) * U
    c2 = math.sqrt(K * W) * U * M
    r = (math.sqrt(lim) + c2) / (1.0 - c1)
    return r * r


def fma32(a, b, c):
    # a * b is exact in double for FP32 a, b; one rounding to FP32 after the add
    return np.float32(float(a) * float(b) + float(c))


def emulate(x, lo, hi, W, form):
    """The kernel's FP32 coarse bound of series x against envelope (lo, hi)."""
    n, d = x.shape
    S = n // W
    sc = np.float32(math.sqrt(W))
    acc = np.float32(0.0)
    for s in range(S):
        seg = x[s * W:(s + 1) * W].astype(np.float64)
        mean = (seg.sum(0) / W).astype(np.float32) * sc
        blo = lo[s * W:(s + 1) * W].min(0).astype(np.float32) * sc
        bhi = hi[s * W:(s + 1) * W].max(0).astype(np.float32) * sc
        box = np.float32(0.0)
        for k in range(d):
            e = max(np.float32(blo[k] - mean[k]), np.float32(mean[k] - bhi[k]), np.float32(0.0))
            box = fma32(e, e, box)
        if form == 0:
            acc = np.float32(acc + box)
        else:
            acc = max(acc, np.float32(box * np.float32(1.0 / W)))
    return float(acc)


def exact(x, lo, hi, W, form):
    """The same bound in FP64 from the unrounded means."""
    n, d = x.shape
    S = n // W
    terms = []
    for s in range(S):
        mean = x[s * W:(s + 1) * W].astype(np.float64).mean(0)
        blo = lo[s * W:(s + 1) * W].astype(np.float64).min(0)
        bhi = hi[s * W:(s + 1) * W].astype(np.float64).max(0)
        e = np.maximum(np.maximum(blo - mean, mean - bhi), 0.0)
        terms.append(float(np.sum(e * e)))
    return sum(W * t for t in terms) if form == 0 else max(terms)


@pytest.mark.parametrize("W,d", [(4, 3), (16, 8), (64, 16)])
@pytest.mark.parametrize("form", [0, 1])
def test_fp32_coarse_bound_stays_within_the_widened_limit(W, d, form):
    rng = np.random.default_rng(100 * W + d + form)
    n = 4 * W + 7
    for _ in range(20):
        offset = float(rng.choice([0.0, 1e3, 3e4]))
        x = (np.cumsum(rng.standard_normal((n, d)), 0) + offset).astype(np.float32)
        q = (np.cumsum(rng.standard_normal((n, d)), 0) + offset
             + rng.uniform(0.0, 4.0)).astype(np.float32)
        r = int(0.1 * n)
        lo = np.stack([q[max(0, i - r):i + r + 1].min(0) for i in range(n)])
        hi = np.stack([q[max(0, i - r):i + r + 1].max(0) for i in range(n)])
        M = float(max(np.abs(x).max(), np.abs(q).max()))
        K = (n // W) * d if form == 0 else d
        Wm = W if form == 0 else 1
        got = emulate(x, lo, hi, W, form)
        ref = exact(x, lo, hi, W, form)
        assert got <= coarse_limit(ref, K, Wm, M), (W, d, form, offset, got, ref)
