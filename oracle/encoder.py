"""FP64 reference of the learned proposal's encoder (forward, loss, backward).

TEST INFRASTRUCTURE ONLY (used by the tests to check the GPU encoder's
gradients); it shares no code with the CUDA library.

Network: three convolutions (kernel 5, same padding, 16 -> 64 -> 64 -> 64
channels, bias, ReLU), mean over the series' positions, linear 64 -> 64.
Predicted distance ||e_a - e_b||^2; loss mean over pairs of
(prediction - target)^2.  With ``bf16=True`` the evaluation rounds to BF16 at
the points where the GPU stores BF16 (the input, the convolution weights,
every convolution output, and the gradient of every convolution's
pre-activation), so that the GPU (FP32 accumulation) and this FP64 version
see the same operands; with ``bf16=False`` it is the exact network, used for
finite-difference checks.

Parameter layout (flat float array): W1 [5][16][64], b1 [64], W2 [5][64][64],
b2, W3 [5][64][64], b3, Wl [64][64] (in x out), bl [64].
"""
from __future__ import annotations

import numpy as np

CIN, C, E, K = 16, 64, 64, 5
SHAPES = [("W1", (K, CIN, C)), ("b1", (C,)), ("W2", (K, C, C)), ("b2", (C,)),
          ("W3", (K, C, C)), ("b3", (C,)), ("Wl", (C, E)), ("bl", (E,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 (ties to even) via FP32, back to float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_same(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """out[t, co] = sum_k sum_ci x[t + k - 2, ci] w[k, ci, co], zero outside."""
    n = x.shape[0]
    xp = np.zeros((n + K - 1, x.shape[1]))
    xp[2:2 + n] = x
    out = np.zeros((n, w.shape[2]))
    for k in range(K):
        out += xp[k:k + n] @ w[k]
    return out


def conv_same_transpose(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient of conv_same with respect to its input."""
    n = dy.shape[0]
    dx = np.zeros((n, w.shape[1]))
    for k in range(K):
        # x[s] feeds out[t] with t = s - k + 2
        for s in range(n):
            t = s - k + 2
            if 0 <= t < n:
                dx[s] += w[k] @ dy[t]
    return dx


def conv_same_wgrad(x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    n = x.shape[0]
    xp = np.zeros((n + K - 1, x.shape[1]))
    xp[2:2 + n] = x
    return np.stack([xp[k:k + n].T @ dy for k in range(K)])


def forward(flat, series, bf16: bool = True):
    """Embeddings [n, 64] and the cache the backward needs."""
    p = unflatten(flat)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    ws = [r(p["W1"]), r(p["W2"]), r(p["W3"])]
    bs = [p["b1"], p["b2"], p["b3"]]
    cache, emb = [], []
    for s in series:
        s = np.asarray(s, dtype=np.float64)
        x0 = np.zeros((s.shape[0], CIN))
        x0[:, :s.shape[1]] = s
        acts = [r(x0)]
        for w, b in zip(ws, bs):
            acts.append(r(np.maximum(conv_same(acts[-1], w) + b, 0.0)))
        h = acts[-1].mean(axis=0)
        emb.append(h @ p["Wl"] + p["bl"])
        cache.append((acts, h))
    return np.array(emb), (cache, ws)


def loss_and_grad(flat, series, pa, pb, targets, bf16: bool = True):
    """Mean loss and its gradient (flat) for the pairs (pa[i], pb[i])."""
    p = unflatten(flat)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    e, (cache, ws) = forward(flat, series, bf16)
    n_pairs = len(pa)
    de = np.zeros_like(e)
    loss = 0.0
    for a, b, t in zip(pa, pb, targets):
        diff = e[a] - e[b]
        res = float(diff @ diff) - float(t)
        loss += res * res / n_pairs
        g = 2.0 * res / n_pairs * 2.0 * diff
        de[a] += g
        de[b] -= g
    grads = {name: np.zeros(shape) for name, shape in SHAPES}
    for i, (acts, h) in enumerate(cache):
        grads["Wl"] += np.outer(h, de[i])
        grads["bl"] += de[i]
        dh = p["Wl"] @ de[i]
        n = acts[0].shape[0]
        dz = r(np.where(acts[3] > 0, np.tile(dh / n, (n, 1)), 0.0))
        for layer in (3, 2, 1):
            grads[f"W{layer}"] += conv_same_wgrad(acts[layer - 1], dz)
            grads[f"b{layer}"] += dz.sum(axis=0)
            if layer > 1:
                da = conv_same_transpose(dz, ws[layer - 1])
                dz = r(np.where(acts[layer - 1] > 0, da, 0.0))
    return loss, flatten(grads)


def init_params(d: int, seed: int = 0) -> np.ndarray:
    """He-normal weights (fan-in), zero biases; input coordinates >= d unused."""
    rng = np.random.default_rng(seed)
    p = {name: np.zeros(shape) for name, shape in SHAPES}
    p["W1"] = rng.standard_normal((K, CIN, C)) * np.sqrt(2.0 / (K * d))
    p["W1"][:, d:, :] = 0.0
    p["W2"] = rng.standard_normal((K, C, C)) * np.sqrt(2.0 / (K * C))
    p["W3"] = rng.standard_normal((K, C, C)) * np.sqrt(2.0 / (K * C))
    p["Wl"] = rng.standard_normal((C, E)) * np.sqrt(2.0 / C)
    return flatten(p)
