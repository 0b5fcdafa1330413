"""GPU parity: every kernel of the scan, through the C-ABI, against the FP64
oracle on the same seeded inputs.

Tolerances (FP32 kernels vs the FP64 oracle): DTW 1e-5 relative, DK 1e-6
relative, LB_Box 1e-5 relative (sum) / 1e-6 (max).  k-NN id sets must be
identical, ties broken by id.
"""
import numpy as np
import pytest

import oracle
from synthdata import make_workload

pytestmark = pytest.mark.gpu

DTW_TOL = 1e-5
DK_TOL = 1e-6


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


def f32(x):
    return float(np.float32(x))


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_knn(ids, dist, oids, odist, kind, k):
    ids = np.asarray(ids)
    dist = np.asarray(dist, dtype=np.float64)
    tol = DTW_TOL if kind == 0 else DK_TOL
    for q in range(ids.shape[0]):
        assert set(ids[q][:k].tolist()) == set(oids[q][:k].tolist()), (q, ids[q], oids[q])
        fin = np.isfinite(odist[q])
        np.testing.assert_allclose(dist[q][fin], odist[q][fin], rtol=tol, atol=1e-30)
        # order: ascending by (distance, id) of the exact values
        order = sorted(range(k), key=lambda j: (odist[q][j], oids[q][j]))
        assert list(ids[q][:k]) == [int(oids[q][j]) for j in order]


# ---------------------------------------------------------------------------
# components

@pytest.mark.parametrize("d", [1, 3, 5])
@pytest.mark.parametrize("r", [0, 2, 9])
def test_envelope(kw, d, r):
    rng = np.random.default_rng(10 * d + r)
    t = rng.standard_normal((37, d)).astype(np.float32)
    for length in (37, 45):
        lo, hi = kw.envelope(cuda(t), r, length)
        olo, ohi = oracle.envelope(t, r, length)
        np.testing.assert_array_equal(lo.cpu().numpy(), olo.astype(np.float32))
        np.testing.assert_array_equal(hi.cpu().numpy(), ohi.astype(np.float32))


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 16])
@pytest.mark.parametrize("form", [0, 1])
def test_lb_box(kw, d, form):
    w = make_workload(n_series=300, n_queries=2, d=d, length_range=(40, 70), n_classes=4,
                      seed=d)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    band = 0.1
    for qi in range(2):
        q = w.query(qi)
        got = db.lb_box(cuda(q), band, form).cpu().numpy().astype(np.float64)
        for c in range(w.n_series):
            x = w.series(c)
            r = oracle.band_radius(len(q), len(x), f32(band))
            if abs(len(q) - len(x)) > r:
                assert got[c] == np.inf
                continue
            # the scan bounds series c against the envelope of the query
            # computed with the bucket's radius, which is at least c's own
            exp = oracle.lb_box(x, q, r, form)
            assert got[c] <= exp * (1 + 1e-5) + 1e-6
    db.close()


def test_lb_box_equal_lengths_exact(kw):
    w = make_workload(n_series=257, n_queries=3, d=3, length=64, n_classes=4, seed=11)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    for form in (0, 1):
        for qi in range(3):
            q = w.query(qi)
            got = db.lb_box(cuda(q), 0.1, form).cpu().numpy().astype(np.float64)
            r = oracle.band_radius(64, 64, f32(0.1))
            exp = np.array([oracle.lb_box(w.series(c), q, r, form) for c in range(w.n_series)])
            np.testing.assert_allclose(got, exp, rtol=1e-5 if form == 0 else 1e-6, atol=1e-6)
    db.close()


@pytest.mark.parametrize("form", [0, 1])
def test_greedy_bound(kw, form):
    w = make_workload(n_series=400, n_queries=2, d=3, length=48, n_classes=4, seed=12)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    agree = 0
    total = 0
    for qi in range(2):
        q = w.query(qi)
        got = db.greedy_ub(cuda(q), 0.1, form).cpu().numpy().astype(np.float64)
        r = oracle.band_radius(48, 48, f32(0.1))
        for c in range(w.n_series):
            x = w.series(c)
            exact = oracle.dk(q, x, r) if form == 0 else oracle.dtw(q, x, r)
            g = oracle.gdk(q, x, r) if form == 0 else oracle.greedy_dtw(q, x, r)
            tol = DK_TOL if form == 0 else DTW_TOL
            assert got[c] >= exact * (1 - tol)          # an upper bound, always
            total += 1
            agree += abs(got[c] - g) <= tol * g + 1e-6   # the same walk, almost always
    assert agree >= 0.98 * total
    db.close()


@pytest.mark.parametrize("d", [1, 2, 3, 7, 16])
@pytest.mark.parametrize("kind", [0, 1])
def test_pairwise(kw, d, kind):
    w = make_workload(n_series=120, n_queries=0, d=d, length_range=(20, 90), n_classes=3,
                      seed=20 + d)
    rng = np.random.default_rng(d)
    pa = rng.integers(0, 120, 300)
    pb = rng.integers(0, 120, 300)
    band = 0.2
    o32, o64 = kw.pairwise(cuda(w.db), cuda(w.db_off), cuda(w.db), cuda(w.db_off), cuda(pa),
                           cuda(pb), band=band, distance=kind, fp64=True)
    exp = oracle.pairwise(w.db, w.db_off, w.db, w.db_off, pa, pb, band=f32(band), kind=kind)
    got32 = o32.cpu().numpy().astype(np.float64)
    got64 = o64.cpu().numpy()
    fin = np.isfinite(exp)
    assert np.all(np.isinf(got32[~fin])) and np.all(np.isinf(got64[~fin]))
    np.testing.assert_allclose(got32[fin], exp[fin], rtol=DTW_TOL if kind == 0 else DK_TOL)
    np.testing.assert_allclose(got64[fin], exp[fin], rtol=1e-13)


@pytest.mark.parametrize("band", [0.02, 0.1, 0.3, 1.0])
@pytest.mark.parametrize("kind", [0, 1])
def test_pairwise_bands_span_variants(kw, band, kind):
    """Bands from r=2 to unconstrained: every lanes-per-pair shape is used."""
    w = make_workload(n_series=64, n_queries=0, d=3, length=200, n_classes=3, seed=30)
    pa = np.arange(64)
    pb = (np.arange(64) * 7 + 3) % 64
    o32, _ = kw.pairwise(cuda(w.db), cuda(w.db_off), cuda(w.db), cuda(w.db_off), cuda(pa),
                         cuda(pb), band=band, distance=kind)
    exp = oracle.pairwise(w.db, w.db_off, w.db, w.db_off, pa, pb, band=f32(band), kind=kind)
    np.testing.assert_allclose(o32.cpu().numpy(), exp, rtol=DTW_TOL if kind == 0 else DK_TOL)


# ---------------------------------------------------------------------------
# the scan

def run_scan(kw, w, *, k, band, kind, seed=0, host=False, **kw_args):
    db = kw.KnnDB(cuda(w.db), w.db_off)
    q = w.q if host else cuda(w.q)
    res = db.scan(q, w.q_off, k=k, band=band, distance=kind, seed=seed, stats=True, **kw_args)
    db.close()
    out = [np.asarray(x.cpu()) if hasattr(x, "cpu") else x for x in res[:-1]]
    return out, res[-1]


@pytest.mark.parametrize("kind", [0, 1])
def test_scan_tiny_config(kw, kind):
    """d=2, 1,000 series of length 64, 10 queries, k=1, band 10%, seed 0."""
    w = make_workload(n_series=1000, n_queries=10, d=2, length=64, n_classes=5, seed=0)
    (ids, dist), st = run_scan(kw, w, k=1, band=0.1, kind=kind)
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind, k=1)
    check_knn(ids, dist, oids, odist, kind, 1)
    assert st["dp_calls"] > 0


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("k,band", [(1, 0.05), (10, 0.05), (10, 0.1)])
@pytest.mark.parametrize("seed", [0, 3])
def test_scan_scale_shape(kw, kind, k, band, seed):
    """d=3 length 256 at reduced N: spans many warp tiles plus a ragged tail."""
    w = make_workload(n_series=3001, n_queries=12, d=3, length=256, n_classes=20, seed=1)
    (ids, dist), st = run_scan(kw, w, k=k, band=band, kind=kind, seed=seed)
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(band), kind=kind, k=k)
    check_knn(ids, dist, oids, odist, kind, k)
    if seed == 3:
        assert st["seeds"] == 12 * max(64, 4 * k)


@pytest.mark.parametrize("kind", [0, 1])
def test_scan_uneven_lengths(kw, kind):
    w = make_workload(n_series=1500, n_queries=6, d=4, length_range=(50, 300), n_classes=8,
                      seed=5)
    (ids, dist), _ = run_scan(kw, w, k=5, band=0.1, kind=kind)
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind, k=5)
    check_knn(ids, dist, oids, odist, kind, 5)


@pytest.mark.parametrize("d", [1, 5, 8, 12, 16])
def test_scan_dimensions(kw, d):
    w = make_workload(n_series=700, n_queries=4, d=d, length=60, n_classes=6, seed=40 + d,
                      correlated=d >= 8)
    for kind in (0, 1):
        (ids, dist), _ = run_scan(kw, w, k=3, band=0.1, kind=kind)
        oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind, k=3)
        check_knn(ids, dist, oids, odist, kind, 3)


@pytest.mark.parametrize("kind", [0, 1])
def test_eps_nn(kw, kind):
    w = make_workload(n_series=2000, n_queries=5, d=3, length=80, n_classes=5, seed=7)
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind, k=40)
    eps = f32(np.median(odist[:, 25]))
    db = kw.KnnDB(cuda(w.db), w.db_off)
    ids, dist, cnt = db.scan(cuda(w.q), w.q_off, k=0, eps=eps, eps_capacity=128, band=0.1,
                             distance=kind)
    db.close()
    e_ids, e_dist, e_cnt = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind,
                                      k=0, eps=eps, cap=128)
    ids, dist, cnt = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()
    np.testing.assert_array_equal(cnt, e_cnt)
    for q in range(5):
        c = int(cnt[q])
        assert list(ids[q, :c]) == list(e_ids[q, :c])
        np.testing.assert_allclose(dist[q, :c], e_dist[q, :c], rtol=DTW_TOL if kind == 0 else DK_TOL)


@pytest.mark.parametrize("kind", [0, 1])
def test_eps_nn_large_capacity(kw, kind):
    """eps-NN with more than 8,192 results per query (global-memory merge
    sort of the result lists).  The result set and counts equal the oracle's;
    each reported distance agrees with the oracle's for that id; rows are in
    the order of the reported values, and no two entries are inverted by more
    than the tolerance of the exact values."""
    import torch
    w = make_workload(n_series=24_000, n_queries=3, d=2, length=48, n_classes=4, seed=17)
    band = f32(0.1)
    tol = DTW_TOL if kind == 0 else DK_TOL
    # eps at the median distance of query 0: about half the database per query
    sample = oracle.knn(w.db[: w.db_off[2001]], w.db_off[:2001], w.query(0), [0, 48],
                        band=band, kind=kind, k=2000)[1]
    eps = f32(np.median(sample))
    cap = 24_000
    e_ids, e_dist, e_cnt = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=band, kind=kind, k=0,
                                      eps=eps, cap=cap)
    assert e_cnt.min() > 8192
    db = kw.KnnDB(cuda(w.db), w.db_off)
    ids, dist, cnt = db.scan(cuda(w.q), w.q_off, k=0, eps=eps, eps_capacity=cap, band=0.1,
                             distance=kind)
    ids, dist, cnt = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()
    np.testing.assert_array_equal(cnt, e_cnt)
    for q in range(3):
        c = int(cnt[q])
        exact = dict(zip(e_ids[q, :c].tolist(), e_dist[q, :c].tolist()))
        got = ids[q, :c].tolist()
        assert set(got) == set(exact)
        ex = np.array([exact[i] for i in got])
        np.testing.assert_allclose(dist[q, :c], ex, rtol=tol, atol=1e-30)
        # reported distances never decrease; exact values are inverted by no
        # more than the tolerance (DK: distinct squares may round to one float)
        assert np.all(np.diff(dist[q, :c]) >= 0)
        assert np.all(ex[1:] >= ex[:-1] * (1 - 2 * tol))
        assert np.all(ids[q, c:] == -1) and np.all(np.isinf(dist[q, c:]))
    # capacity overflow on the same path: true counts and valid entries
    small = 9000
    o = (torch.empty((3, small), dtype=torch.int64, device="cuda"),
         torch.empty((3, small), dtype=torch.float32, device="cuda"),
         torch.empty(3, dtype=torch.int64, device="cuda"))
    with pytest.raises(kw.KnnError) as e:
        db.scan(cuda(w.q), w.q_off, k=0, eps=eps, eps_capacity=small, band=0.1, distance=kind,
                out=o)
    assert e.value.status == 5
    db.close()
    # counts of overflowing rows bound the true sizes from above, exceeding
    # them only by results within the FP32 band of eps that were not stored
    band_cnt = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=band, kind=kind, k=0,
                          eps=eps * (1 + 1e-4), cap=cap)[2]
    got_cnt = o[2].cpu().numpy()
    assert np.all(got_cnt >= e_cnt) and np.all(got_cnt <= band_cnt)
    oi = o[0].cpu().numpy()
    for q in range(3):
        exact = set(e_ids[q, : int(e_cnt[q])].tolist())
        assert set(x for x in oi[q].tolist() if x >= 0) <= exact


def test_seed_modes_and_graph_give_identical_results(kw):
    w = make_workload(n_series=2500, n_queries=8, d=3, length=96, n_classes=10, seed=8)
    for kind in (0, 1):
        base, _ = run_scan(kw, w, k=7, band=0.1, kind=kind, seed=0)
        for kwargs in (dict(seed=2), dict(seed=3), dict(seed=3, seed_count=5),
                       dict(seed=3, use_graph=True), dict(seed=0, use_graph=True),
                       dict(seed=0, query_batch=3), dict(seed=0, host=True)):
            other, _ = run_scan(kw, w, k=7, band=0.1, kind=kind, **kwargs)
            np.testing.assert_array_equal(base[0], other[0])
            np.testing.assert_array_equal(base[1], other[1])


def test_graph_replay_is_stable(kw):
    w = make_workload(n_series=1200, n_queries=6, d=2, length=64, n_classes=5, seed=9)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    q = cuda(w.q)
    first = db.scan(q, w.q_off, k=4, band=0.1, distance=0, use_graph=True)
    for _ in range(3):
        again = db.scan(q, w.q_off, k=4, band=0.1, distance=0, use_graph=True)
        assert (again[0] == first[0]).all() and (again[1] == first[1]).all()
    db.close()


def test_edge_cases(kw):
    rng = np.random.default_rng(3)
    # series of length 1, a query of length 1, unconstrained band, k = N
    lens = np.array([1, 2, 1, 3, 5, 1, 4])
    off = np.concatenate([[0], np.cumsum(lens)])
    db_pts = rng.standard_normal((off[-1], 2)).astype(np.float32)
    q = rng.standard_normal((1, 2)).astype(np.float32)
    for kind in (0, 1):
        db = kw.KnnDB(cuda(db_pts), off)
        ids, dist = db.scan(cuda(q), np.array([0, 1]), k=7, band=1.0, distance=kind)
        db.close()
        oids, odist = oracle.knn(db_pts, off, q, np.array([0, 1]), band=1.0, kind=kind, k=7)
        check_knn(ids.cpu().numpy(), dist.cpu().numpy(), oids, odist, kind, 7)


def test_infeasible_lengths_are_never_returned(kw):
    w = make_workload(n_series=200, n_queries=2, d=2, length_range=(10, 200), n_classes=3, seed=2)
    (ids, dist), st = run_scan(kw, w, k=20, band=0.05, kind=0)
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.05), kind=0, k=20)
    for q in range(2):
        fin = np.isfinite(odist[q])
        assert list(ids[q][fin]) == list(oids[q][fin])
        assert np.all(ids[q][~fin] == -1) and np.all(np.isinf(dist[q][~fin]))
    assert st["band_infeasible"] > 0


def test_duplicates_ordered_by_id(kw):
    w = make_workload(n_series=300, n_queries=1, d=3, length=50, n_classes=4, seed=13)
    db_pts = np.concatenate([w.db, w.db[:50], w.db[:50], w.db[:50]])
    off = np.concatenate([w.db_off, w.db_off[-1] + np.array([50, 100, 150])])
    q = w.db[:50].copy()
    for kind in (0, 1):
        db = kw.KnnDB(cuda(db_pts), off)
        ids, dist = db.scan(cuda(q), np.array([0, 50]), k=4, band=0.1, distance=kind)
        db.close()
        assert list(ids.cpu().numpy()[0]) == [0, 300, 301, 302]
        assert np.all(dist.cpu().numpy()[0] == 0)


def test_invalid_arguments(kw):
    w = make_workload(n_series=50, n_queries=1, d=2, length=20, n_classes=2, seed=1)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    for bad in (dict(k=51), dict(k=-1), dict(band=0.0), dict(band=float("nan")),
                dict(k=0, eps=1.0, eps_capacity=0), dict(distance=7)):
        args = dict(k=1, band=0.1, distance=0)
        args.update(bad)
        with pytest.raises(kw.KnnError) as e:
            db.scan(cuda(w.q), w.q_off, **args)
        assert e.value.status == 1
    bad_q = w.q.copy()
    bad_q[3, 1] = np.nan
    with pytest.raises(kw.KnnError):
        db.scan(cuda(bad_q), w.q_off, k=1, band=0.1)
    with pytest.raises(kw.KnnError):
        kw.KnnDB(cuda(w.db), np.array([0, 5, 5, 20]))      # empty series
    db.close()


def test_scan_simple_single_query_form(kw):
    """knn_scan_simple: one host query against host series given by lengths."""
    w = make_workload(n_series=400, n_queries=1, d=3, length=40, n_classes=4, seed=14)
    lens = w.db_lengths()
    for kind in (0, 1):
        ids, dist = kw.scan_simple(w.query(0), w.db, lens, d=3, band=0.1, k=5, distance=kind)
        oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind, k=5)
        check_knn(ids[None], dist[None], oids, odist, kind, 5)


@pytest.mark.parametrize("kind", [0, 1])
def test_every_dp_shape_gives_identical_results(kw, kind):
    """The autotuner may pick any compiled shape: all must return the same."""
    w = make_workload(n_series=1500, n_queries=6, d=3, length=128, n_classes=8, seed=15)
    band, k = 0.1, 5
    r = oracle.band_radius(128, 128, f32(band))
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(band), kind=kind, k=k)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    shapes = []
    for P in kw.dp_shapes(3):
        G = 1
        while G * P < r + 1:
            G *= 2
        for g in (G, 2 * G):
            if g <= 32:
                shapes.append((P, g))
    assert len(shapes) >= 4
    for seed in (0, 3):
        for P, G in shapes:
            db.set_dp_shape(kind, r, 128, P, G)
            assert db.get_dp_shape(kind, r, 128) == (P, G)
            ids, dist = db.scan(cuda(w.q), w.q_off, k=k, band=band, distance=kind, seed=seed)
            check_knn(ids.cpu().numpy(), dist.cpu().numpy(), oids, odist, kind, k)
    with pytest.raises(kw.KnnError):
        db.set_dp_shape(kind, r, 128, 3, 32)          # P=3 is not compiled
    with pytest.raises(kw.KnnError):
        db.set_dp_shape(kind, r, 128, 2, 1)           # G*P < r+1
    db.close()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d", [8, 16])
@pytest.mark.parametrize("band", [0.1, 0.3])
def test_wide_point_dp_shapes(kw, kind, d, band):
    """d >= 8 with 8 or more lanes per pair stages query rows and series
    columns in shared memory: every such shape returns the oracle's result."""
    w = make_workload(n_series=600, n_queries=4, d=d, length=160, n_classes=6, seed=50 + d,
                      correlated=True)
    k = 4
    r = oracle.band_radius(160, 160, f32(band))
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(band), kind=kind, k=k)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    shapes = []
    for P in kw.dp_shapes(d):
        G = 1
        while G * P < r + 1:
            G *= 2
        shapes += [(P, g) for g in (G, 2 * G) if 8 <= g <= 32]
    assert {g for _, g in shapes} >= ({8, 16, 32} if band == 0.1 else {32})
    for seed in (kw.SEED_NONE, kw.SEED_LB):
        for P, G in shapes:
            db.set_dp_shape(kind, r, 160, P, G)
            ids, dist = db.scan(cuda(w.q), w.q_off, k=k, band=band, distance=kind, seed=seed)
            check_knn(ids.cpu().numpy(), dist.cpu().numpy(), oids, odist, kind, k)
    db.close()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d,lengths,nq", [(3, (40, 300), 21), (16, (300, 700), 9)])
def test_lb_tiles_and_windows_give_identical_results(kw, kind, d, lengths, nq):
    """LB_Box with 4, 8 or 16 queries per pass, whole envelopes or windows of
    them (several sizes, ragged last window, a partial query tile): every
    variant bounds the same way, so every scan returns the oracle's result."""
    w = make_workload(n_series=700 if d == 3 else 300, n_queries=nq, d=d, length_range=lengths,
                      n_classes=6, seed=31 + d)
    band, k = 0.1, 4
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(band), kind=kind, k=k)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    assert db.get_lb_tile(kind) == (0, 0, 0)
    ref = None
    for qt, win, comp in [(q, w_, 0) for q in (4, 8, 16) for w_ in (0, 1, 5, 64)] + \
            [(q, 0, c) for q in (4, 16) for c in (1, 2)]:
        if True:
            db.set_lb_tile(kind, qt, win, comp)
            assert db.get_lb_tile(kind) == (qt, win, comp)
            for seed in (kw.SEED_GREEDY, kw.SEED_LB, kw.SEED_NONE):
                ids, dist = db.scan(cuda(w.q), w.q_off, k=k, band=band, distance=kind, seed=seed)
                ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
                check_knn(ids, dist, oids, odist, kind, k)
                if ref is None:
                    ref = (ids, dist)
                assert (ids == ref[0]).all() and (dist == ref[1]).all()
    for bad in ((kind, 5, 0, 0), (kind, 16, -1, 0), (2, 16, 0, 0), (kind, 16, 0, 3)):
        with pytest.raises(kw.KnnError):
            db.set_lb_tile(*bad)
    db.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_lb_compaction_gives_identical_results(kw, kind):
    """The compacting LB_Box kernel (survivor queues between checkpoints) must
    bound and queue exactly as the plain one: one bucket of 5,000 series, so
    that CTAs walk several batches and the queues fill past 256 entries; with
    no seed threshold (every series survives every checkpoint) and with one."""
    w = make_workload(n_series=5000, n_queries=24, d=3, length=128, n_classes=6, seed=41)
    band, k = 0.1, 5
    oids, odist = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(band), kind=kind, k=k)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    ref = None
    for comp in (1, 2, 0):
        for qt in (16, 8):
            db.set_lb_tile(kind, qt, 0, comp)
            for seed in (kw.SEED_NONE, kw.SEED_GREEDY):
                ids, dist, st = db.scan(cuda(w.q), w.q_off, k=k, band=band, distance=kind,
                                        seed=seed, stats=True)
                ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
                check_knn(ids, dist, oids, odist, kind, k)
                if ref is None:
                    ref = (ids, dist)
                assert (ids == ref[0]).all() and (dist == ref[1]).all()
                assert st["pairs"] == 24 * 5000
    db.close()


def test_autotune_and_cache(kw, tmp_path):
    w = make_workload(n_series=3000, n_queries=16, d=3, length_range=(60, 200), n_classes=8,
                      seed=16)
    cache = str(tmp_path / "shapes.json")
    db = kw.KnnDB(cuda(w.db), w.db_off)
    base = db.scan(cuda(w.q), w.q_off, k=5, band=0.1, distance=0, seed=3)
    db.autotune(cuda(w.q), w.q_off, k=5, band=0.1, distance=0, cache_path=cache)
    tuned = db.scan(cuda(w.q), w.q_off, k=5, band=0.1, distance=0, seed=3)
    assert (tuned[0] == base[0]).all() and (tuned[1] == base[1]).all()
    import json
    entries = json.load(open(cache))["dp_shapes"]
    assert len(entries) == db.info()["n_buckets"]
    assert all(e["P"] * e["G"] >= e["r"] + 1 for e in entries)
    db.close()
    # a fresh database reuses the cached shapes without re-timing
    db2 = kw.KnnDB(cuda(w.db), w.db_off)
    db2.autotune(cuda(w.q), w.q_off, k=5, band=0.1, distance=0, cache_path=cache)
    e = entries[0]
    assert db2.get_dp_shape(0, e["r"], e["n"]) == (e["P"], e["G"])
    db2.close()


# ---------------------------------------------------------------------------
# coarse first stage of the LB_Box cascade (segment boxes)

@pytest.mark.parametrize("d,L", [(1, 50), (2, 50), (3, 50), (5, 50), (8, 96), (12, 96),
                                 (16, 96), (8, 256), (16, 300)])
@pytest.mark.parametrize("form", [0, 1])
def test_lb_seg_component(kw, d, L, form):
    """knn_lb_seg against the oracle's segment-box bound (same W, same band
    radius), and never above knn_lb_box; W = 4 for d < 8, 16 or 64 (series
    of at least 256 points) for d >= 8."""
    rng = np.random.default_rng(70 + d + 10 * form)
    w = make_workload(n_series=300, n_queries=2, d=d, length=L, n_classes=4, seed=60 + d)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    _, W = db.get_lb_cascade(0)
    assert W == (4 if d < 8 else 64 if L >= 256 else 16)
    band = 0.1
    r = oracle.band_radius(L, L, f32(band))
    for qi in range(2):
        q = w.query(qi)
        got = db.lb_seg(cuda(q), band, form).cpu().numpy().astype(np.float64)
        box = db.lb_box(cuda(q), band, form).cpu().numpy().astype(np.float64)
        exp = np.array([oracle.lb_seg(w.series(c), q, r, W, form) for c in range(300)])
        scale = max(1.0, float(exp.max()))
        np.testing.assert_allclose(got, exp, rtol=1e-5, atol=1e-6 * scale)
        assert np.all(got <= box * (1 + 1e-5) + 1e-6 * scale)
    db.close()


@pytest.mark.parametrize("d,lengths,L", [(3, None, 80), (3, (40, 200), 80), (8, (64, 160), 80),
                                         (16, None, 128), (16, None, 256)])
def test_coarse_stage_gives_identical_results(kw, d, lengths, L):
    """Scans with the coarse first stage (default) and without it return the
    same rows bit for bit, for DTW and DK, k-NN under every seeding and
    eps-NN; the stage runs and prunes (16-point segments at d = 16, L = 128;
    64-point ones at L = 256)."""
    w = make_workload(n_series=2500, n_queries=12, d=d, length=L, length_range=lengths,
                      n_classes=8, seed=90 + d)
    db = kw.KnnDB(cuda(w.db), w.db_off)
    q = cuda(w.q)
    enc = kw.Encoder(d, seed=3)
    enc.attach(db)
    for kind in (kw.DTW, kw.DK):
        for seed in (kw.SEED_LEARNED, kw.SEED_GREEDY, kw.SEED_NONE):
            db.set_lb_cascade(kind, 0)
            on = db.scan(q, w.q_off, k=6, band=0.1, distance=kind, seed=seed, stats=True)
            db.set_lb_cascade(kind, 1)
            off = db.scan(q, w.q_off, k=6, band=0.1, distance=kind, seed=seed, stats=True)
            np.testing.assert_array_equal(on[0].cpu().numpy(), off[0].cpu().numpy())
            np.testing.assert_array_equal(on[1].cpu().numpy(), off[1].cpu().numpy())
            assert on[2]["lb_kernels"] & 16 and not off[2]["lb_kernels"] & 16
            assert off[2]["lb_coarse_pruned"] == 0
            assert on[2]["lb_pruned"] == off[2]["lb_pruned"]
            if seed != kw.SEED_NONE:  # without seeding the threshold is +inf at LB time
                assert on[2]["lb_coarse_pruned"] > 0
                assert on[2]["lb_points"] < off[2]["lb_points"]
        if lengths is None:
            oi, od = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=f32(0.1), kind=kind, k=6)
            db.set_lb_cascade(kind, 0)
            ids, dist = db.scan(q, w.q_off, k=6, band=0.1, distance=kind, seed=kw.SEED_LEARNED)
            check_knn(ids.cpu().numpy(), dist.cpu().numpy(), oi, od, kind, 6)
        eps = float(np.float32(np.median(on[1].cpu().numpy()[:, 3])))
        res = []
        for coarse in (0, 1):
            db.set_lb_cascade(kind, coarse)
            res.append(db.scan(q, w.q_off, k=0, eps=eps, eps_capacity=2500, band=0.1,
                               distance=kind))
        for a, b in zip(res[0], res[1]):
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    enc.close()
    db.close()
