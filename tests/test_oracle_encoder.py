"""Pins for the FP64 encoder reference: the convolution against NumPy's
correlate, its two gradients against finite differences, and the whole
backward against finite differences of the loss."""
import numpy as np
import pytest

from oracle import encoder as enc


def test_conv_same_matches_numpy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((20, 1))
    w = rng.standard_normal((5, 1, 1))
    out = enc.conv_same(x, w)[:, 0]
    # out[t] = sum_k x[t+k-2] w[k]: a 'same' cross-correlation
    ref = np.correlate(np.pad(x[:, 0], 2), w[:, 0, 0], mode="valid")
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_conv_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((9, 3))
    w = rng.standard_normal((5, 3, 4))
    dy = rng.standard_normal((9, 4))
    f = lambda xx, ww: float(np.sum(enc.conv_same(xx, ww) * dy))
    dx = enc.conv_same_transpose(dy, w)
    dw = enc.conv_same_wgrad(x, dy)
    h = 1e-6
    for (i, j) in [(0, 0), (4, 2), (8, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j] += h
        xm[i, j] -= h
        assert dx[i, j] == pytest.approx((f(xp, w) - f(xm, w)) / (2 * h), rel=1e-6, abs=1e-8)
    for (k, i, j) in [(0, 0, 0), (2, 1, 3), (4, 2, 1)]:
        wp, wm = w.copy(), w.copy()
        wp[k, i, j] += h
        wm[k, i, j] -= h
        assert dw[k, i, j] == pytest.approx((f(x, wp) - f(x, wm)) / (2 * h), rel=1e-6, abs=1e-8)


def test_backward_by_finite_differences():
    rng = np.random.default_rng(2)
    series = [rng.standard_normal((int(n), 3)) for n in (7, 11, 9, 6)]
    flat = enc.init_params(3, seed=3)
    flat[enc.N_PARAMS - 64:] = rng.standard_normal(64) * 0.1        # non-zero bl
    pa, pb = [0, 1, 2], [1, 3, 0]
    targets = [0.5, 2.0, 1.0]
    loss, grad = enc.loss_and_grad(flat, series, pa, pb, targets, bf16=False)
    h = 1e-6
    idx = rng.choice(enc.N_PARAMS, 40, replace=False)
    idx = [i for i in idx if not (i < 5 * 16 * 64 and (i // 64) % 16 >= 3)]  # unused inputs
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = enc.loss_and_grad(fp, series, pa, pb, targets, bf16=False)
        lm, _ = enc.loss_and_grad(fm, series, pa, pb, targets, bf16=False)
        assert grad[i] == pytest.approx((lp - lm) / (2 * h), rel=2e-4, abs=1e-7), i


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -3.14159, 0.0])
    r = enc.round_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0                     # tie -> even
    assert r[2] == 1.0 + 4 * 2 ** -8                       # tie -> even (up)
    assert abs(r[3] + 3.140625) < 1e-12 and r[4] == 0.0
