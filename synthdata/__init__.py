"""Seeded synthetic workloads for the k-NN / eps-NN time-warping scan.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no distance, bound or envelope).  Both the FP64 oracle's
tests and the GPU path consume what it returns.

Recipe (class-structured warped random walks, standing in for the RAM/CBF
generators and the real data sets of Section 5, which are not available):

* class template: a random walk ``cumsum(N(0,1))`` per dimension;
  for correlated channels (motion-capture-like) channel ``j`` is
  ``0.9 * x[j-1] + sqrt(0.19) * w[j]`` with ``w[j]`` an independent walk;
* instance: the template resampled by linear interpolation at a random
  monotone piecewise-linear time warp with 8 segments whose slopes are
  U[0.5, 1.5] (renormalised to map [0,1] onto [0,1]), plus N(0, sigma^2)
  noise, sigma = 0.1;
* queries are fresh instances of random classes.

Series are stored point-major: ``points[off[i]:off[i+1], :]`` is series ``i``
with shape ``[len_i, d]``, float32.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import os
from concurrent.futures import ThreadPoolExecutor
from typing import Optional

import numpy as np

N_WARP_SEGMENTS = 8


@dataclass
class Workload:
    """A database plus a query batch."""

    d: int
    db: np.ndarray            # [sum(len), d] float32
    db_off: np.ndarray        # [N+1] int64, point offsets
    db_labels: np.ndarray     # [N] int32
    q: np.ndarray             # [sum(qlen), d] float32
    q_off: np.ndarray         # [Q+1] int64
    q_labels: np.ndarray      # [Q] int32
    meta: dict = field(default_factory=dict)

    @property
    def n_series(self) -> int:
        return int(self.db_off.shape[0] - 1)

    @property
    def n_queries(self) -> int:
        return int(self.q_off.shape[0] - 1)

    def series(self, i: int) -> np.ndarray:
        return self.db[self.db_off[i]:self.db_off[i + 1]]

    def query(self, i: int) -> np.ndarray:
        return self.q[self.q_off[i]:self.q_off[i + 1]]

    def db_lengths(self) -> np.ndarray:
        return np.diff(self.db_off)

    def q_lengths(self) -> np.ndarray:
        return np.diff(self.q_off)


def _templates(rng: np.random.Generator, n_classes: int, length: int, d: int,
               correlated: bool) -> np.ndarray:
    walks = np.cumsum(rng.standard_normal((n_classes, length, d)), axis=1)
    if not correlated:
        return walks
    out = np.empty_like(walks)
    out[:, :, 0] = walks[:, :, 0]
    a, b = 0.9, np.sqrt(0.19)
    for j in range(1, d):
        out[:, :, j] = a * out[:, :, j - 1] + b * walks[:, :, j]
    return out


def _warp_knots(rng: np.random.Generator, count: int) -> np.ndarray:
    """Cumulative warp values at the 9 knots of an 8-segment monotone warp."""
    slopes = rng.uniform(0.5, 1.5, size=(count, N_WARP_SEGMENTS))
    cum = np.concatenate([np.zeros((count, 1)), np.cumsum(slopes, axis=1)], axis=1)
    return cum / cum[:, -1:]


def _resample(templ_flat: np.ndarray, lt: int, classes: np.ndarray, knots: np.ndarray,
              lens: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """Instances of the templates of ``classes`` (series i has lens[i] points):
    point p of series i takes the template at the warped position of
    u = p / (lens[i] - 1), linearly interpolated, plus its noise.
    templ_flat is [n_classes * lt, d] float32; noise is [sum(lens), d] float32
    and is overwritten with the result, which is returned."""
    lens = np.asarray(lens, dtype=np.int64)
    sid = np.repeat(np.arange(lens.shape[0]), lens)                    # series of each point
    start = np.zeros(lens.shape[0], dtype=np.int64)
    np.cumsum(lens[:-1], out=start[1:])
    p = np.arange(sid.shape[0], dtype=np.int64) - start[sid]
    u = p / np.maximum(lens[sid] - 1, 1)
    # piecewise-linear warp: knot x positions are uniform in [0,1]
    seg = np.minimum((u * N_WARP_SEGMENTS).astype(np.int64), N_WARP_SEGMENTS - 1)
    frac = u * N_WARP_SEGMENTS - seg
    w = knots[sid, seg] * (1.0 - frac) + knots[sid, seg + 1] * frac
    tau = np.clip(w, 0.0, 1.0) * (lt - 1)
    i0 = np.minimum(np.floor(tau).astype(np.int64), lt - 2 if lt > 1 else 0)
    f = (tau - i0).astype(np.float32)[:, None]
    base = classes.astype(np.int64)[sid] * lt
    g0 = templ_flat[base + i0]                                         # [points, d]
    g1 = templ_flat[base + np.minimum(i0 + 1, lt - 1)]
    g1 -= g0
    g1 *= f
    noise += g0
    noise += g1
    return noise


# Every block of BLOCK consecutive series (database or queries) draws its
# classes, warps, lengths and noise from its own stream, keyed by (seed,
# role, block index), so that a database prefix or the queries can be drawn
# without the rest and blocks can be drawn in parallel.
BLOCK = 1024
_DB, _QUERIES, _TEMPLATES = 1, 2, 0


def _stream(seed: int, role: int, block: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed,
                                                                      spawn_key=(role, block))))


def _block_header(g: np.random.Generator, count: int, n_classes: int, length,
                  length_range):
    classes = g.integers(0, n_classes, size=count).astype(np.int32)
    knots = _warp_knots(g, count)
    if length_range is None:
        lens = np.full(count, int(length), dtype=np.int64)
    else:
        lens = g.integers(length_range[0], length_range[1] + 1, size=count).astype(np.int64)
    return classes, knots, lens


def _draw_set(seed: int, role: int, count: int, templ_flat: np.ndarray, lt: int, d: int,
              n_classes: int, length, length_range, noise_sigma: float, threads: int):
    """Series ``0 .. count-1`` of one role: (points [sum(len), d], offsets, classes)."""
    nb = (count + BLOCK - 1) // BLOCK
    heads = []
    for b in range(nb):
        c = min(BLOCK, count - b * BLOCK)
        h = _block_header(_stream(seed, role, b), BLOCK, n_classes, length, length_range)
        heads.append(tuple(x[:c] for x in h))
    lens = np.concatenate([h[2] for h in heads]) if nb else np.zeros(0, np.int64)
    classes = np.concatenate([h[0] for h in heads]) if nb else np.zeros(0, np.int32)
    off = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    pts = np.empty((int(off[-1]), d), dtype=np.float32)

    def fill(b):
        g = _stream(seed, role, b)
        c = min(BLOCK, count - b * BLOCK)
        # the header is drawn for a whole block, so a partial last block
        # draws the same values as the full one
        cl, kn, ln = _block_header(g, BLOCK, n_classes, length, length_range)
        cl, kn, ln = cl[:c], kn[:c], ln[:c]
        noise = g.standard_normal((int(ln.sum()), d), dtype=np.float32)
        noise *= np.float32(noise_sigma)
        pts[off[b * BLOCK]: off[b * BLOCK + c]] = _resample(templ_flat, lt, cl, kn, ln, noise)

    if nb:
        with ThreadPoolExecutor(max_workers=max(1, min(threads, nb))) as ex:
            list(ex.map(fill, range(nb)))
    return pts, off, classes


def make_workload(*, n_series: int, n_queries: int, d: int, length=64,
                  n_classes: int = 5, seed: int = 0, noise_sigma: float = 0.1,
                  correlated: bool = False, length_range: Optional[tuple] = None,
                  template_length: Optional[int] = None,
                  threads: Optional[int] = None) -> Workload:
    """Draw a seeded workload.

    ``length`` fixes every series length; ``length_range=(lo, hi)`` draws each
    length uniformly from the integers in [lo, hi] instead (both database and
    queries).  Series i of the database depends only on (seed, i) and the
    recipe, so a smaller ``n_series`` gives a prefix of the larger database;
    the queries do not depend on ``n_series``.
    """
    lt = template_length or (length_range[1] if length_range else length)
    templ = _templates(_stream(seed, _TEMPLATES), n_classes, lt, d, correlated)
    templ_flat = np.ascontiguousarray(templ.reshape(-1, d), dtype=np.float32)
    threads = threads or min(32, os.cpu_count() or 1)
    db, db_off, db_lab = _draw_set(seed, _DB, n_series, templ_flat, lt, d, n_classes, length,
                                   length_range, noise_sigma, threads)
    q, q_off, q_lab = _draw_set(seed, _QUERIES, n_queries, templ_flat, lt, d, n_classes, length,
                                length_range, noise_sigma, threads)
    return Workload(
        d=d, db=db, db_off=db_off, db_labels=db_lab, q=q, q_off=q_off, q_labels=q_lab,
        meta=dict(seed=seed, n_classes=n_classes, noise_sigma=noise_sigma,
                  correlated=correlated, length=length, length_range=length_range),
    )


@dataclass
class LongSeries:
    """One long series and a batch of queries for subsequence search."""

    d: int
    t: np.ndarray             # [n, d] float32
    q: np.ndarray             # [sum(qlen), d] float32
    q_off: np.ndarray         # [Q+1] int64
    meta: dict = field(default_factory=dict)


def make_long_series(*, n: int, n_queries: int, d: int, q_length: int, n_classes: int = 20,
                     seed: int = 0, noise_sigma: float = 0.1, batch: int = 4096) -> LongSeries:
    """A long series made of consecutive class instances (the recipe of
    make_workload, lengths U[q_length/2, 2 q_length]) and queries that are
    fresh instances of length q_length (stand-in for querying one long ECG
    recording)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lt = 2 * q_length
    templ = _templates(rng, n_classes, lt, d, False)
    tflat = np.ascontiguousarray(templ.reshape(-1, d), dtype=np.float32)
    chunks, total, last = [], 0, None
    while total < n:
        lens = rng.integers(q_length // 2, 2 * q_length + 1, size=batch)
        classes = rng.integers(0, n_classes, size=batch).astype(np.int32)
        knots = _warp_knots(rng, batch)
        nz = (rng.standard_normal((int(lens.sum()), d)) * noise_sigma).astype(np.float32)
        chunk = _resample(tflat, lt, classes, knots, lens, nz)
        if last is not None:          # continue from where the previous chunk ended
            chunk = chunk - chunk[0] + last
        last = chunk[-1]
        chunks.append(chunk.astype(np.float32))
        total += chunk.shape[0]
    pieces_all = np.concatenate(chunks)
    t = pieces_all[:n].astype(np.float32)
    qc = rng.integers(0, n_classes, size=n_queries).astype(np.int32)
    qk = _warp_knots(rng, n_queries)
    nz = (rng.standard_normal((n_queries * q_length, d)) * noise_sigma).astype(np.float32)
    q = _resample(tflat, lt, qc, qk, np.full(n_queries, q_length), nz)
    q_off = np.arange(n_queries + 1, dtype=np.int64) * q_length
    return LongSeries(d=d, t=t, q=q, q_off=q_off,
                      meta=dict(seed=seed, n_classes=n_classes, q_length=q_length))


LONG_SERIES = {
    # one series of 1,000,000 points, d=1, 1,024 queries of 256 points
    "subseq_d1_T1M_m256": dict(n=1_000_000, n_queries=1024, d=1, q_length=256, seed=5),
    # d=3, 1,000,000 points, 1,024 queries of 128 points
    "subseq_d3_T1M_m128": dict(n=1_000_000, n_queries=1024, d=3, q_length=128, seed=6),
}


# Named workloads (sizes of the scan's benchmark configurations).
WORKLOADS = {
    # d=2, 1,000 series of length 64, 10 queries, 5 classes, seed 0
    "tiny_d2_n1k_L64": dict(n_series=1000, n_queries=10, d=2, length=64, n_classes=5, seed=0),
    # d=3, 100,000 series of length 256, 1,000 queries, 20 classes
    "scale_d3_n100k_L256": dict(n_series=100_000, n_queries=1000, d=3, length=256,
                                n_classes=20, seed=1),
    # 200,000 series, lengths U[50,1000], 256 queries; one data set per d in 3..8
    **{f"uneven_d{d}_n200k_L50_1000": dict(n_series=200_000, n_queries=256, d=d,
                                           length_range=(50, 1000), n_classes=20,
                                           seed=2 + d) for d in range(3, 9)},
    # d=3, 1,000,000 series of length 128, 1,000 queries, 50 classes
    "learned_d3_n1M_L128": dict(n_series=1_000_000, n_queries=1000, d=3, length=128,
                                n_classes=50, seed=3),
    # d=16 correlated channels (AR(1), rho=0.9), 500,000 series of length 512
    "highdim_d16_n500k_L512": dict(n_series=500_000, n_queries=1000, d=16, length=512,
                                   n_classes=50, seed=4, correlated=True),
}


def named(name: str, **overrides) -> Workload:
    """Build a named workload; ``overrides`` may shrink it (e.g. n_series)."""
    kw = dict(WORKLOADS[name])
    kw.update(overrides)
    return make_workload(**kw)
