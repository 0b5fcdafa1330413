"""FP64 oracle for the exact k-NN / eps-NN time-warping scan.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product path never does.  It shares no
code with the CUDA library.  The arithmetic lives in ``oracle.c`` (plain C,
double precision); this module compiles it with gcc on first use and marshals
numpy arrays through ctypes.

Each wrapper cites the passage of Bachmann & Freytag (arXiv 1811.11076) that it
follows; see ``oracle.c`` for the definitions written out.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTW = 0
DK = 1

_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_band_radius.restype = C.c_int64
            L.orc_band_radius.argtypes = [C.c_int64, C.c_int64, C.c_double]
            for name in ("orc_dtw", "orc_dk"):
                f = getattr(L, name)
                f.restype = C.c_double
                f.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64]
            L.orc_envelope.restype = None
            L.orc_envelope.argtypes = [_d, C.c_int64, C.c_int, C.c_int64, C.c_int64, _d, _d]
            L.orc_lb_keogh_1d.restype = C.c_double
            L.orc_lb_keogh_1d.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int64]
            L.orc_lb_box.restype = C.c_double
            L.orc_lb_box.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64, C.c_int]
            L.orc_lb_seg.restype = C.c_double
            L.orc_lb_seg.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64, C.c_int64,
                                     C.c_int]
            L.orc_lb_sigma_min.restype = C.c_double
            L.orc_lb_sigma_min.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64]
            L.orc_greedy.restype = C.c_double
            L.orc_greedy.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64,
                                     C.c_double, C.c_int]
            L.orc_sub_distance.restype = C.c_double
            L.orc_sub_distance.argtypes = [C.c_int, _d, C.c_int64, _d, C.c_int64, C.c_int, _i64]
            L.orc_sub_ends.restype = C.c_int64
            L.orc_sub_ends.argtypes = [C.c_int, _d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64,
                                       _d, _i64]
            L.orc_sub_sparse_dk.restype = C.c_double
            L.orc_sub_sparse_dk.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_double,
                                            _i64, _i64]
            L.orc_sub_gdk.restype = C.c_double
            L.orc_sub_gdk.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_double, _i64]
            for name in ("orc_sparse_dk", "orc_dtw_abandon"):
                f = getattr(L, name)
                f.restype = C.c_double
                f.argtypes = [_d, C.c_int64, _d, C.c_int64, C.c_int, C.c_int64, C.c_double, _i64]
            L.orc_knn.restype = C.c_int
            L.orc_knn.argtypes = [_d, _i64, C.c_int64, _d, _i64, C.c_int64, C.c_int, C.c_double,
                                  C.c_int, C.c_int64, C.c_double, C.c_int64, C.c_int, C.c_int,
                                  _i64, _d, _i64, _i64]
            L.orc_pairwise.restype = C.c_int
            L.orc_pairwise.argtypes = [_d, _i64, _d, _i64, _i64, _i64, C.c_int64, C.c_int,
                                       C.c_double, C.c_int, C.c_int, _d]
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return a


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def band_radius(m: int, n: int, band: float) -> int:
    """r = floor(band * max(m, n)); band >= 1 is unconstrained (Section 2.2)."""
    return int(lib().orc_band_radius(m, n, band))


def _pair_args(s, t):
    s = _f64(s)
    t = _f64(t)
    assert s.shape[1] == t.shape[1]
    return s, t, s.shape[0], t.shape[0], s.shape[1]


def dtw(s, t, r: int) -> float:
    """Banded DTW, sum of squared Euclidean point costs (Section 2.1, 2.2)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_dtw(_p(s), m, _p(t), n, d, r)


def dk(s, t, r: int) -> float:
    """Banded dog-keeper distance, max of Euclidean point costs (Section 2.1)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_dk(_p(s), m, _p(t), n, d, r)


def distance(kind: int, s, t, r: int) -> float:
    return dk(s, t, r) if kind == DK else dtw(s, t, r)


def envelope(t, r: int, length: int | None = None):
    """Per-dimension band envelope l, u of ``t`` (Sections 2.3 and 3)."""
    t = _f64(t)
    n, d = t.shape
    length = n if length is None else length
    lo = np.empty((length, d))
    hi = np.empty((length, d))
    lib().orc_envelope(_p(t), n, d, r, length, _p(lo), _p(hi))
    return lo, hi


def lb_keogh_1d(s, t, r: int) -> float:
    """LB_Keogh of 1-D series (Section 2.3), envelope taken on ``t``."""
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64).ravel())
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).ravel())
    return lib().orc_lb_keogh_1d(_p(s), s.shape[0], _p(t), t.shape[0], r)


def lb_box(s, t, r: int, form: int = 0) -> float:
    """LB_Box (Section 3, Eq. 1): form 0 sums, form 1 takes the max (squared)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_lb_box(_p(s), m, _p(t), n, d, r, form)


def lb_seg(s, t, r: int, W: int, form: int = 0) -> float:
    """LB_Box over segment boxes of W points (the cascade's coarse stage,
    Section 3 Eq. 1 on coarsened boxes): W * squared distance of each whole
    segment's mean of s to the box holding its envelope boxes, summed (form
    0) or the max of the squared distances (form 1)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_lb_seg(_p(s), m, _p(t), n, d, r, W, form)


def lb_sigma_min(s, t, r: int) -> float:
    """LB_Sigma-min (Section 3)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_lb_sigma_min(_p(s), m, _p(t), n, d, r)


def gdk(s, t, r: int, eps: float = float("inf")) -> float:
    """Greedy dog-keeper upper bound (Section 4.1, Algorithm 1)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_greedy(_p(s), m, _p(t), n, d, r, eps, 0)


def greedy_dtw(s, t, r: int, eps: float = float("inf")) -> float:
    """Sum of squared costs along the greedy path of Algorithm 1 (DTW upper bound)."""
    s, t, m, n, d = _pair_args(s, t)
    return lib().orc_greedy(_p(s), m, _p(t), n, d, r, eps, 1)


def sparse_dk(s, t, r: int, eps: float):
    """Sparse DK, whole match (Section 4.2, Algorithm 3); returns (value, cells)."""
    s, t, m, n, d = _pair_args(s, t)
    cells = C.c_int64(0)
    v = lib().orc_sparse_dk(_p(s), m, _p(t), n, d, r, eps, C.byref(cells))
    return v, cells.value


def sub_distance(kind: int, s, t):
    """Subsequence search, plain definition (free-start/free-end DP, no band):
    min over subsequences T[a..b] of DTW (kind 0, sum of squared costs) or DK
    (kind 1, Euclidean) of S against T[a..b].  Returns (value, end b)."""
    s, t, m, n, d = _pair_args(s, t)
    end = C.c_int64(-1)
    v = lib().orc_sub_distance(kind, _p(s), m, _p(t), n, d, C.byref(end))
    return v, end.value


def sub_ends(kind: int, s, t, k: int):
    """The k best end columns of subsequence search (the free-start recursion
    of sub_distance): the k smallest (D(m, b), b) over every column b, ordered
    by (value, b).  Returns (values[k], ends[k]), padded with +inf / -1."""
    s, t, m, n, d = _pair_args(s, t)
    val = np.empty(k)
    end = np.empty(k, dtype=np.int64)
    lib().orc_sub_ends(kind, _p(s), m, _p(t), n, d, k, _p(val), _p(end, _i64))
    return val, end


def sub_sparse_dk(s, t, eps: float):
    """Algorithm 3 with SUB = true; returns (value or +inf above eps, end, cells)."""
    s, t, m, n, d = _pair_args(s, t)
    end, cells = C.c_int64(-1), C.c_int64(0)
    v = lib().orc_sub_sparse_dk(_p(s), m, _p(t), n, d, eps, C.byref(end), C.byref(cells))
    return v, end.value, cells.value


def sub_gdk(s, t, eps: float = float("inf")):
    """Greedy dog-keeper for subsequence search (Algorithm 2); returns (bound, end)."""
    s, t, m, n, d = _pair_args(s, t)
    end = C.c_int64(-1)
    v = lib().orc_sub_gdk(_p(s), m, _p(t), n, d, eps, C.byref(end))
    return v, end.value


def dtw_abandon(s, t, r: int, eps: float):
    """DTW with row-minimum early abandoning (Section 4); returns (value, cells)."""
    s, t, m, n, d = _pair_args(s, t)
    cells = C.c_int64(0)
    v = lib().orc_dtw_abandon(_p(s), m, _p(t), n, d, r, eps, C.byref(cells))
    return v, cells.value


def knn(db, db_off, queries, q_off, *, band: float, kind: int, k: int = 1,
        eps: float = float("inf"), cap: int = 0, method: bool = False,
        threads: int | None = None, with_stats: bool = False):
    """Exact k-NN (k > 0) or eps-NN (k == 0) in FP64 (Section 1 query types).

    method=False: every distance, sorted by (distance, id).
    method=True:  the paper's pruned scan (LB_Box cascade, GDK pre-pass,
                  sparse DK, DTW early abandoning), which must give the same.
    Returns (ids, dists) for k-NN, (ids, dists, counts) for eps-NN, plus a
    per-query stats array [lb_pruned, dp_calls, dp_abandoned, cells, ub_calls]
    when with_stats.
    """
    db = _f64(db)
    queries = _f64(queries)
    d = db.shape[1]
    db_off = np.ascontiguousarray(db_off, dtype=np.int64)
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    N = db_off.shape[0] - 1
    nq = q_off.shape[0] - 1
    width = k if k > 0 else cap
    ids = np.full((nq, max(width, 1)), -1, dtype=np.int64)
    dist = np.full((nq, max(width, 1)), np.inf)
    counts = np.zeros(max(nq, 1), dtype=np.int64)
    stats = np.zeros((max(nq, 1), 5), dtype=np.int64)
    threads = threads or os.cpu_count() or 1
    lib().orc_knn(_p(db), _p(db_off, _i64), N, _p(queries), _p(q_off, _i64), nq, d, band,
                  kind, k, eps, cap, int(method), threads, _p(ids, _i64), _p(dist),
                  _p(counts, _i64), _p(stats, _i64))
    ids, dist, counts, stats = ids[:, :width], dist[:, :width], counts[:nq], stats[:nq]
    out = (ids, dist) if k > 0 else (ids, dist, counts)
    return out + (stats,) if with_stats else out


def pairwise(a, a_off, b, b_off, pa, pb, *, band: float, kind: int,
             threads: int | None = None) -> np.ndarray:
    """FP64 distances of the pairs (a[pa[i]], b[pb[i]])."""
    a = _f64(a)
    b = _f64(b)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    out = np.empty(pa.shape[0])
    lib().orc_pairwise(_p(a), _p(a_off, _i64), _p(b), _p(b_off, _i64), _p(pa, _i64),
                       _p(pb, _i64), pa.shape[0], a.shape[1], band, kind,
                       threads or os.cpu_count() or 1, _p(out))
    return out
