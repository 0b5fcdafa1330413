"""knn_pairwise_noalloc: the pair programs for callers who cannot let the
library allocate device memory.  Its results must match those of
knn_pairwise (which allocates its own scratch) on two calls in a row; it must
also reject inputs beyond its fixed scratch with a clear error.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from synthdata import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_11076_gb300 as kw
    from paper_1811_11076_gb300 import build
    build.build()
    kw.lib()
    return kw


def _call(kw, a, a_off, b, b_off, pa, pb, d, band, max_len, kind, out):
    import torch
    return kw.lib().knn_pairwise_noalloc(
        a.data_ptr(), a_off.data_ptr(), a_off.numel() - 1, b.data_ptr(), b_off.data_ptr(),
        b_off.numel() - 1, pa.data_ptr(), pb.data_ptr(), pa.numel(), d, C.c_float(band),
        max_len, kind, out.data_ptr(), torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_matches_allocating_pairwise(kw, kind):
    """Calls in a row (d = 3, 5, 12 with its zero-padded coordinates, 1): each
    result equals knn_pairwise's and the FP64 oracle's within the tolerance,
    and once the first call has loaded the library's array no call changes
    the device's free memory."""
    import torch
    import oracle
    tol = 1e-5 if kind == 0 else 1e-6
    free_before = []
    for call, (d, seed) in enumerate([(3, 1), (5, 2), (12, 3), (1, 4)]):
        wa = make_workload(n_series=150, n_queries=0, d=d, length_range=(30, 120), n_classes=4,
                           seed=100 + seed)
        wb = make_workload(n_series=220, n_queries=0, d=d, length_range=(30, 120), n_classes=4,
                           seed=200 + seed)
        rng = np.random.default_rng(seed)
        n = 2000
        pa_h, pb_h = rng.integers(0, 150, n), rng.integers(0, 220, n)
        pa, pb = torch.from_numpy(pa_h).cuda(), torch.from_numpy(pb_h).cuda()
        a, a_off = torch.from_numpy(wa.db).cuda(), torch.from_numpy(wa.db_off).cuda()
        b, b_off = torch.from_numpy(wb.db).cuda(), torch.from_numpy(wb.db_off).cuda()
        band = 0.1
        ref, _ = kw.pairwise(a, a_off, b, b_off, pa, pb, band=band, distance=kind)
        out = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call(kw, a, a_off, b, b_off, pa, pb, d, band, 120, kind, out)
        assert st == 0, kw.lib().knn_last_error()
        torch.cuda.synchronize()
        free_before.append((free0, torch.cuda.mem_get_info()[0]))
        got, exp = out.cpu().numpy(), ref.cpu().numpy()
        fin = np.isfinite(exp)
        assert np.array_equal(np.isinf(got), ~fin), call
        np.testing.assert_allclose(got[fin], exp[fin], rtol=tol, atol=0)
        orc = oracle.pairwise(wa.db, wa.db_off, wb.db, wb.db_off, pa_h, pb_h,
                              band=float(np.float32(band)), kind=kind)
        assert np.array_equal(np.isfinite(orc), fin), call
        np.testing.assert_allclose(got[fin], orc[fin], rtol=tol, atol=0)
    # no device memory is taken by any call after the first
    for f0, f1 in free_before[1:]:
        assert f0 == f1


def test_noalloc_refuses_a_stream_under_capture(kw):
    import torch
    w = make_workload(n_series=8, n_queries=0, d=2, length=30, n_classes=2, seed=7)
    a, a_off = torch.from_numpy(w.db).cuda(), torch.from_numpy(w.db_off).cuda()
    idx = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    assert _call(kw, a, a_off, a, a_off, idx, idx, 2, 0.1, 30, 0, out) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g.capture_begin()
        st = _call(kw, a, a_off, a, a_off, idx, idx, 2, 0.1, 30, 0, out)
        g.capture_end()
    torch.cuda.synchronize()
    assert st == 1 and b"captured" in kw.lib().knn_last_error()
    assert _call(kw, a, a_off, a, a_off, idx, idx, 2, 0.1, 30, 0, out) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(kw):
    import torch
    w = make_workload(n_series=10, n_queries=0, d=2, length=40, n_classes=2, seed=5)
    a, a_off = torch.from_numpy(w.db).cuda(), torch.from_numpy(w.db_off).cuda()
    out = torch.empty(70000, dtype=torch.float32, device="cuda")
    many = torch.zeros(70000, dtype=torch.int64, device="cuda")
    st = _call(kw, a, a_off, a, a_off, many, many, 2, 0.1, 40, 0, out)
    assert st == 1 and b"65536" in kw.lib().knn_last_error()
    # a series longer than the stated max_len is an error, not a silent clamp
    few = torch.zeros(4, dtype=torch.int64, device="cuda")
    st = _call(kw, a, a_off, a, a_off, few, few, 2, 0.1, 20, 0, out)
    assert st == 1 and b"max_len" in kw.lib().knn_last_error()
    # total padded floats above the fixed capacity
    big = make_workload(n_series=300, n_queries=0, d=16, length=300, n_classes=2, seed=6)
    ba, bo = torch.from_numpy(big.db).cuda(), torch.from_numpy(big.db_off).cuda()
    st = _call(kw, ba, bo, ba, bo, few, few, 16, 0.1, 300, 0, out)
    assert st == 5 and b"1,048,576" in kw.lib().knn_last_error()
