"""Exact k-NN / eps-NN scan of multi-dimensional time series under banded DTW
and the dog-keeper distance DK, on NVIDIA GB300 (sm_103a).

Method: Bachmann & Freytag, "An Analytical Approach to Improving Time Warping
on Multidimensional Time Series" (arXiv 1811.11076): LB_Box pruning
(Section 3, Eq. 1), GDK upper bounds (Section 4.1, Algorithm 1),
threshold-driven DK (Section 4.2, Algorithm 3), nearest-neighbour search with
an upper-bound pre-pass (Section 4.3).

This module only marshals arguments to the C-ABI of ``libknnwarp.so``
(declared in ``include/knnwarp.h``); every step of the scan runs in the
library's CUDA kernels.  There is no CPU fallback: if the library has not
been built, importing works but every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libknnwarp.so")

DTW = 0
DK = 1
SEED_GREEDY = 0
SEED_LEARNED = 1
SEED_NONE = 2
SEED_LB = 3
SEED_LEARNED_ = SEED_LEARNED

STATUS = {0: "KNN_OK", 1: "KNN_ERR_INVALID", 2: "KNN_ERR_OOM", 3: "KNN_ERR_CUDA",
          4: "KNN_ERR_TIMEOUT", 5: "KNN_ERR_CAPACITY", 6: "KNN_ERR_UNSUPPORTED"}

# every symbol include/knnwarp.h declares
EXPORTS = ("knn_db_create", "knn_db_destroy", "knn_db_info", "knn_scan", "knn_scan_simple",
           "knn_envelope", "knn_lb_box", "knn_greedy_ub", "knn_pairwise", "knn_status_string",
           "knn_last_error", "knn_version", "knn_autotune", "knn_set_dp_shape", "knn_get_dp_shape",
           "knn_dp_shapes", "knn_set_lb_tile", "knn_get_lb_tile", "knn_set_lb_cascade",
           "knn_get_lb_cascade", "knn_lb_seg", "knn_subseq", "knn_subseq_k", "knn_db_create_windows", "knn_subseq_greedy", "knn_pairwise_noalloc", "knn_encoder_num_params", "knn_encoder_create",
           "knn_encoder_destroy", "knn_encoder_train", "knn_encoder_embed", "knn_encoder_attach", "knn_encoder_scores",
           "knn_encoder_params", "knn_encoder_loss_grad", "knn_encoder_save", "knn_encoder_load")


class KnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("k", C.c_int32), ("eps", C.c_float), ("band", C.c_float),
                ("distance", C.c_int32), ("seed_mode", C.c_int32), ("seed_count", C.c_int32),
                ("query_batch", C.c_int32), ("use_graph", C.c_int32),
                ("eps_capacity", C.c_int64), ("profile", C.c_int32), ("reserved", C.c_int32)]


class TrainParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch_pairs", C.c_int32), ("lr", C.c_float),
                ("distance", C.c_int32), ("band", C.c_float), ("seed", C.c_uint64)]


class TrainStats(C.Structure):
    _fields_ = [("first_loss", C.c_double), ("final_loss", C.c_double), ("ms", C.c_double),
                ("pairs", C.c_int64), ("steps", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("band_infeasible", C.c_int64), ("ub_walks", C.c_int64),
                ("seeds", C.c_int64), ("seed_cells", C.c_int64), ("lb_pruned", C.c_int64), ("lb_pruned_late", C.c_int64),
                ("dp_calls", C.c_int64), ("dp_abandoned", C.c_int64), ("dp_cells", C.c_int64),
                ("reranked", C.c_int64), ("lb_points", C.c_int64), ("launches", C.c_int64), ("ms_total", C.c_double),
                ("ms_seed", C.c_double), ("ms_lb", C.c_double), ("ms_dp", C.c_double),
                ("ms_finalize", C.c_double), ("lb_kernels", C.c_int64),
                ("lb_coarse_pruned", C.c_int64), ("lb_segments", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib() -> C.CDLL:
    """Load libknnwarp.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1811_11076_gb300.build` (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, i64p = C.c_void_p, C.c_void_p
    L.knn_db_create.argtypes = [vp, vp, C.c_int64, C.c_int32, vp, C.POINTER(vp)]
    L.knn_db_destroy.argtypes = [vp]
    L.knn_db_create_windows.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32, vp,
                                        C.POINTER(vp)]
    L.knn_db_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                              C.POINTER(C.c_int32)]
    L.knn_scan.argtypes = [vp, vp, vp, C.c_int32, C.POINTER(Params), vp, vp, vp,
                           C.POINTER(Stats), vp]
    L.knn_scan_simple.argtypes = [vp, C.c_int64, vp, vp, C.c_int64, C.c_int32, C.c_float,
                                  C.c_int32, C.c_float, C.c_int32, vp, vp,
                                  C.POINTER(C.c_int64)]
    L.knn_envelope.argtypes = [vp, C.c_int64, C.c_int32, C.c_int64, C.c_int64, vp, vp, vp]
    L.knn_lb_box.argtypes = [vp, vp, C.c_int64, C.c_float, C.c_int32, vp, vp]
    L.knn_greedy_ub.argtypes = [vp, vp, C.c_int64, C.c_float, C.c_int32, vp, vp]
    L.knn_lb_seg.argtypes = [vp, vp, C.c_int64, C.c_float, C.c_int32, vp, vp]
    L.knn_set_lb_cascade.argtypes = [vp, C.c_int32, C.c_int32]
    L.knn_get_lb_cascade.argtypes = [vp, C.c_int32] + [C.POINTER(C.c_int32)] * 2
    L.knn_pairwise.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int64, C.c_int32, C.c_float,
                               C.c_int32, vp, vp, vp]
    L.knn_autotune.argtypes = [vp, vp, vp, C.c_int32, C.POINTER(Params), C.c_char_p, vp]
    L.knn_set_dp_shape.argtypes = [vp] + [C.c_int32] * 5
    L.knn_get_dp_shape.argtypes = [vp] + [C.c_int32] * 3 + [C.POINTER(C.c_int32)] * 2
    L.knn_dp_shapes.argtypes = [C.c_int32, vp, C.c_int32]
    L.knn_subseq.argtypes = [vp, vp, C.c_int32, vp, C.c_int64, C.c_int32, C.c_int32, C.c_float,
                             vp, vp, vp]
    L.knn_subseq_k.argtypes = [vp, vp, C.c_int32, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                               C.c_float, vp, vp, vp]
    L.knn_subseq_greedy.argtypes = [vp, vp, C.c_int32, vp, C.c_int64, C.c_int32, C.c_float, vp,
                                    vp, vp]
    L.knn_set_lb_tile.argtypes = [vp] + [C.c_int32] * 4
    L.knn_get_lb_tile.argtypes = [vp, C.c_int32] + [C.POINTER(C.c_int32)] * 3
    L.knn_pairwise_noalloc.argtypes = [vp, vp, C.c_int64, vp, vp, C.c_int64, vp, vp, C.c_int64,
                                       C.c_int32, C.c_float, C.c_int32, C.c_int32, vp, vp]
    L.knn_encoder_num_params.restype = C.c_int32
    L.knn_encoder_create.argtypes = [C.c_int32, C.c_uint64, C.POINTER(vp)]
    L.knn_encoder_destroy.argtypes = [vp]
    L.knn_encoder_train.argtypes = [vp, vp, C.c_int64, C.POINTER(TrainParams),
                                    C.POINTER(TrainStats), vp]
    L.knn_encoder_embed.argtypes = [vp, vp, vp, C.c_int64, vp, vp]
    L.knn_encoder_attach.argtypes = [vp, vp, vp]
    L.knn_encoder_scores.argtypes = [vp, vp, vp, C.c_int32, vp, vp, vp]
    L.knn_encoder_params.argtypes = [vp, vp, vp]
    L.knn_encoder_loss_grad.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, C.c_int64,
                                        C.POINTER(C.c_float), vp, vp]
    L.knn_encoder_save.argtypes = [vp, C.c_char_p]
    L.knn_encoder_load.argtypes = [C.c_char_p, C.POINTER(vp)]
    for f in EXPORTS:
        if f not in ("knn_status_string", "knn_last_error", "knn_version",
                     "knn_encoder_num_params"):
            getattr(L, f).restype = C.c_int
    L.knn_status_string.restype = C.c_char_p
    L.knn_status_string.argtypes = [C.c_int]
    L.knn_last_error.restype = C.c_char_p
    L.knn_version.restype = C.c_char_p
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise KnnError(status, lib().knn_last_error().decode())


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array (contiguous)."""
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _stream(stream=None) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def _f32(a):
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.float32).contiguous()
    return np.ascontiguousarray(a, dtype=np.float32)


def _i64(a):
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.int64).contiguous()
    return np.ascontiguousarray(a, dtype=np.int64)


class KnnDB:
    """A database of series in the library's device layout (knn_db)."""

    def __init__(self, series, offsets, d: int | None = None, stream=None):
        series = _f32(series)
        offsets = _i64(offsets)
        if d is None:
            d = int(series.shape[1]) if len(series.shape) == 2 else 1
        h = C.c_void_p()
        self._keep = (series, offsets)
        _check(lib().knn_db_create(_ptr(series), _ptr(offsets), int(offsets.shape[0] - 1), int(d),
                                   _stream(stream), C.byref(h)))
        self._h = h
        self._keep = None
        self.d = int(d)
        self.n = int(offsets.shape[0] - 1)

    @classmethod
    def windows(cls, series, m: int, stride: int = 1, stream=None) -> "KnnDB":
        """The windows T[a .. a+m-1] of one long series T [n][d] (a = 0,
        stride, ...): a scan of length-m queries against it is the banded
        subsequence search; result ids are window indices (start = id *
        stride)."""
        series = _f32(series)
        d = int(series.shape[1]) if len(series.shape) == 2 else 1
        n = int(series.shape[0])
        h = C.c_void_p()
        _check(lib().knn_db_create_windows(_ptr(series), n, d, int(m), int(stride),
                                           _stream(stream), C.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        self._keep = None
        self.d = d
        self.n = (n - int(m)) // int(stride) + 1
        return self

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        n, d, b = C.c_int64(), C.c_int32(), C.c_int32()
        _check(lib().knn_db_info(self._h, C.byref(n), C.byref(d), C.byref(b)))
        return {"n_series": n.value, "d": d.value, "n_buckets": b.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().knn_db_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def scan(self, queries, q_offsets, *, k: int = 1, eps: float = 0.0, band: float = 0.1,
             distance: int = DTW, seed: int = SEED_GREEDY, seed_count: int = 0,
             query_batch: int = 0, use_graph: bool = False, eps_capacity: int = 0,
             out=None, stream=None, stats: bool = False, profile: bool = False):
        """Exact k-NN (k > 0) or eps-NN (k == 0).  Inputs and outputs may be
        host (numpy / CPU tensors) or device (CUDA tensors).  Returns
        (ids, dist) for k-NN, (ids, dist, counts) for eps-NN, plus a stats
        dict if requested."""
        queries = _f32(queries)
        q_offsets = _i64(q_offsets)
        nq = int(q_offsets.shape[0] - 1)
        width = k if k > 0 else eps_capacity
        if out is None:
            dev = hasattr(queries, "is_cuda") and queries.is_cuda
            if dev:
                import torch
                ids = torch.empty((nq, width), dtype=torch.int64, device=queries.device)
                dist = torch.empty((nq, width), dtype=torch.float32, device=queries.device)
                counts = torch.empty(nq, dtype=torch.int64, device=queries.device)
            else:
                ids = np.empty((nq, width), dtype=np.int64)
                dist = np.empty((nq, width), dtype=np.float32)
                counts = np.empty(nq, dtype=np.int64)
        else:
            ids, dist, counts = out
        p = Params(k=k, eps=eps, band=band, distance=distance, seed_mode=seed,
                   seed_count=seed_count, query_batch=query_batch, use_graph=int(use_graph),
                   eps_capacity=eps_capacity, profile=int(profile))
        st = Stats()
        _check(lib().knn_scan(self._h, _ptr(queries), _ptr(q_offsets), nq, C.byref(p), _ptr(ids),
                              _ptr(dist), _ptr(counts), C.byref(st), _stream(stream)))
        res = (ids, dist) if k > 0 else (ids, dist, counts)
        return res + (st.as_dict(),) if stats else res

    def autotune(self, queries, q_offsets, *, k: int = 10, band: float = 0.1,
                 distance: int = DTW, seed: int = 3, cache_path: str | None = None,
                 stream=None):
        """Time every compiled DP shape per length bucket; keep the fastest."""
        queries = _f32(queries)
        q_offsets = _i64(q_offsets)
        p = Params(k=k, band=band, distance=distance, seed_mode=seed)
        _check(lib().knn_autotune(self._h, _ptr(queries), _ptr(q_offsets),
                                  int(q_offsets.shape[0] - 1), C.byref(p),
                                  cache_path.encode() if cache_path else None, _stream(stream)))

    def set_dp_shape(self, distance: int, r: int, n: int, P: int, G: int):
        _check(lib().knn_set_dp_shape(self._h, distance, r, n, P, G))

    def set_lb_tile(self, distance: int, qtile: int = 0, window_chunks: int = 0,
                    compaction: int = 0):
        """Queries per LB_Box pass, envelope window and compaction (0: automatic)."""
        _check(lib().knn_set_lb_tile(self._h, distance, qtile, window_chunks, compaction))

    def get_lb_tile(self, distance: int):
        q, w, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().knn_get_lb_tile(self._h, distance, C.byref(q), C.byref(w), C.byref(c)))
        return q.value, w.value, c.value

    def set_lb_cascade(self, distance: int, coarse: int = 0):
        """Coarse first LB stage (segment boxes): 0 automatic, 1 never."""
        _check(lib().knn_set_lb_cascade(self._h, distance, coarse))

    def get_lb_cascade(self, distance: int):
        """(setting, segment width W)."""
        c, w = C.c_int32(), C.c_int32()
        _check(lib().knn_get_lb_cascade(self._h, distance, C.byref(c), C.byref(w)))
        return c.value, w.value

    def lb_seg(self, query, band: float, form: int = 0, stream=None):
        """Coarse (segment box) bound of every series (device tensor out)."""
        import torch
        query = _f32(query)
        out = torch.empty(self.n, dtype=torch.float32, device="cuda")
        _check(lib().knn_lb_seg(self._h, _ptr(query), int(query.shape[0]), band, form, _ptr(out),
                                _stream(stream)))
        return out

    def get_dp_shape(self, distance: int, r: int, n: int):
        P, G = C.c_int32(), C.c_int32()
        _check(lib().knn_get_dp_shape(self._h, distance, r, n, C.byref(P), C.byref(G)))
        return P.value, G.value

    def lb_box(self, query, band: float, form: int = 0, stream=None):
        """LB_Box of every series against the query envelope (device tensor out)."""
        import torch
        query = _f32(query)
        out = torch.empty(self.n, dtype=torch.float32, device="cuda")
        _check(lib().knn_lb_box(self._h, _ptr(query), int(query.shape[0]), band, form, _ptr(out),
                                _stream(stream)))
        return out

    def greedy_ub(self, query, band: float, form: int = 0, stream=None):
        """Greedy (Algorithm 1) upper bound of every series (device tensor out)."""
        import torch
        query = _f32(query)
        out = torch.empty(self.n, dtype=torch.float32, device="cuda")
        _check(lib().knn_greedy_ub(self._h, _ptr(query), int(query.shape[0]), band, form,
                                   _ptr(out), _stream(stream)))
        return out


class Encoder:
    """The learned proposal's 1-D convolutional encoder (knn_encoder)."""

    def __init__(self, d: int = 3, seed: int = 0, _handle=None):
        if _handle is None:
            h = C.c_void_p()
            _check(lib().knn_encoder_create(d, seed, C.byref(h)))
            _handle = h
        self._h = _handle
        self.d = d

    @staticmethod
    def num_params() -> int:
        return int(lib().knn_encoder_num_params())

    @classmethod
    def load(cls, path: str) -> "Encoder":
        h = C.c_void_p()
        _check(lib().knn_encoder_load(path.encode(), C.byref(h)))
        enc = cls(_handle=h)
        enc.d = -1
        return enc

    def save(self, path: str):
        _check(lib().knn_encoder_save(self._h, path.encode()))

    def params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().knn_encoder_params(self._h, out.ctypes.data, None))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.shape[0] == self.num_params()
        _check(lib().knn_encoder_params(self._h, None, flat.ctypes.data))

    def train(self, db: "KnnDB", n_pairs: int, *, epochs: int = 4, batch_pairs: int = 2048,
              lr: float = 1e-3, distance: int = DTW, band: float = 0.1, seed: int = 0,
              stream=None) -> dict:
        tp = TrainParams(epochs=epochs, batch_pairs=batch_pairs, lr=lr, distance=distance,
                         band=band, seed=seed)
        st = TrainStats()
        _check(lib().knn_encoder_train(self._h, db.handle, n_pairs, C.byref(tp), C.byref(st),
                                       _stream(stream)))
        return st.as_dict()

    def embed(self, series, offsets, stream=None):
        import torch
        series = _f32(series)
        offsets = _i64(offsets)
        n = int(offsets.shape[0] - 1)
        out = torch.empty((n, 64), dtype=torch.float32, device="cuda")
        _check(lib().knn_encoder_embed(self._h, _ptr(series), _ptr(offsets), n, _ptr(out),
                                       _stream(stream)))
        return out

    @staticmethod
    def scores(db: "KnnDB", queries, q_offsets, stream=None):
        """Tile-best proposal scores of the encoder attached to db (tensor
        cores): ([nq][tiles] float32, [nq][tiles] int64 series ids)."""
        import torch
        queries = _f32(queries)
        q_offsets = _i64(q_offsets)
        nq = int(q_offsets.shape[0] - 1)
        tiles = (db.n + 63) // 64
        sc = torch.empty((nq, tiles), dtype=torch.float32, device="cuda")
        ids = torch.empty((nq, tiles), dtype=torch.int64, device="cuda")
        _check(lib().knn_encoder_scores(db.handle, _ptr(queries), _ptr(q_offsets), nq, _ptr(sc),
                                        _ptr(ids), _stream(stream)))
        return sc, ids

    def attach(self, db: "KnnDB", stream=None):
        _check(lib().knn_encoder_attach(db.handle, self._h, _stream(stream)))
        db._encoder = self  # keep alive while attached

    def loss_grad(self, series, offsets, pa, pb, targets, stream=None):
        series = _f32(series)
        offsets = _i64(offsets)
        pa, pb = _i64(pa), _i64(pb)
        targets = np.ascontiguousarray(targets, dtype=np.float32)
        loss = C.c_float()
        grad = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().knn_encoder_loss_grad(self._h, _ptr(series), _ptr(offsets),
                                           int(offsets.shape[0] - 1), _ptr(pa), _ptr(pb),
                                           targets.ctypes.data, int(pa.shape[0]),
                                           C.byref(loss), grad.ctypes.data, _stream(stream)))
        return loss.value, grad

    def close(self):
        if getattr(self, "_h", None):
            lib().knn_encoder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def subseq(queries, q_offsets, series, *, distance: int = DK, eps: float = float("inf"),
           greedy: bool = False, k: int = 1, stream=None):
    """Subsequence search of every query against one long series (Section 4.2,
    Algorithm 3 with SUB = true; greedy=True: the Algorithm 2 upper bound).
    queries [sum m][d], q_offsets [nq+1], series [n][d]: host or device.
    Returns (values, ends) on the inputs' device: [nq] for k = 1, else
    [nq][k], the k best end columns by (value, end)."""
    import torch
    queries = _f32(queries)
    q_offsets = _i64(q_offsets)
    series = _f32(series)
    nq = int(q_offsets.shape[0] - 1)
    d = int(series.shape[1]) if series.ndim > 1 else 1
    on_gpu = hasattr(series, "is_cuda") and series.is_cuda
    dev = series.device if on_gpu else torch.device("cpu")
    shape = (nq,) if k == 1 or greedy else (nq, k)
    vals = torch.empty(shape, dtype=torch.float32, device=dev)
    ends = torch.empty(shape, dtype=torch.int64, device=dev)
    if greedy:
        _check(lib().knn_subseq_greedy(_ptr(queries), _ptr(q_offsets), nq, _ptr(series),
                                       int(series.shape[0]), d, eps, _ptr(vals), _ptr(ends),
                                       _stream(stream)))
    elif k == 1:
        _check(lib().knn_subseq(_ptr(queries), _ptr(q_offsets), nq, _ptr(series),
                                int(series.shape[0]), d, distance, eps, _ptr(vals), _ptr(ends),
                                _stream(stream)))
    else:
        _check(lib().knn_subseq_k(_ptr(queries), _ptr(q_offsets), nq, _ptr(series),
                                  int(series.shape[0]), d, distance, k, eps, _ptr(vals),
                                  _ptr(ends), _stream(stream)))
    return vals, ends


def dp_shapes(d: int) -> list[int]:
    """Compiled P values (band cells per lane) for dimensionality d."""
    n = lib().knn_dp_shapes(d, None, 0)
    buf = (C.c_int32 * max(n, 1))()
    lib().knn_dp_shapes(d, C.cast(buf, C.c_void_p), n)
    return list(buf[:n])


def envelope(t, r: int, length: int | None = None, stream=None):
    """Band envelope (lo, hi) of a device series t [n, d] (Sections 2.3, 3)."""
    import torch
    t = _f32(t)
    n, d = int(t.shape[0]), int(t.shape[1])
    length = n if length is None else length
    lo = torch.empty((length, d), dtype=torch.float32, device=t.device)
    hi = torch.empty((length, d), dtype=torch.float32, device=t.device)
    _check(lib().knn_envelope(_ptr(t), n, d, r, length, _ptr(lo), _ptr(hi), _stream(stream)))
    return lo, hi


def pairwise(a, a_off, b, b_off, pa, pb, *, band: float, distance: int, fp64: bool = False,
             fp32: bool = True, stream=None):
    """Banded DTW/DK of pairs (a[pa[i]], b[pb[i]]); device tensors in and out."""
    import torch
    a, b = _f32(a), _f32(b)
    a_off, b_off, pa, pb = _i64(a_off), _i64(b_off), _i64(pa), _i64(pb)
    n = int(pa.shape[0])
    d = int(a.shape[1])
    o32 = torch.empty(n, dtype=torch.float32, device=a.device) if fp32 else None
    o64 = torch.empty(n, dtype=torch.float64, device=a.device) if fp64 else None
    _check(lib().knn_pairwise(_ptr(a), _ptr(a_off), _ptr(b), _ptr(b_off), _ptr(pa), _ptr(pb), n,
                              d, band, distance, _ptr(o32) if fp32 else None,
                              _ptr(o64) if fp64 else None, _stream(stream)))
    return o32, o64


def scan_simple(query, db, lengths, *, d: int, band: float, k: int = 1, eps: float = 0.0,
                distance: int = DTW):
    """knn_scan(query, db, lengths, d, band, k|eps, distance) -> ids, distances."""
    query = _f32(query)
    db = _f32(db)
    lengths = _i64(lengths)
    n = int(lengths.shape[0])
    width = k if k > 0 else min(n, 8192)
    ids = np.empty(width, dtype=np.int64)
    dist = np.empty(width, dtype=np.float32)
    cnt = C.c_int64(0)
    _check(lib().knn_scan_simple(_ptr(query), int(query.shape[0]), _ptr(db), _ptr(lengths), n, d,
                                 band, k, eps, distance, _ptr(ids), _ptr(dist), C.byref(cnt)))
    if k > 0:
        return ids, dist
    c = min(cnt.value, width)
    return ids[:c], dist[:c]
