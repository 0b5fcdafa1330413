"""GPU subsequence search (Algorithm 3 with SUB = true; the free-start DTW;
Algorithm 2) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1811_11076_gb300 as kw_
    kw_.lib()
    return kw_


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def walk_series(rng, n, d):
    return np.cumsum(rng.standard_normal((n, d)), axis=0).astype(np.float32)


TOL = {0: 1e-5, 1: 1e-6}   # relative, DTW / DK (values re-scored in FP64)


def check(kind, q, t, v, end):
    """GPU value within the tolerance of the oracle's (no absolute slack) and
    the same end column (the smallest of equal best values)."""
    ov, oend = oracle.sub_distance(kind, q.astype(np.float64), t.astype(np.float64))
    assert v == pytest.approx(ov, rel=TOL[kind], abs=0), (v, ov)
    assert end == oend, (end, oend, v, ov)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d", [1, 3, 8, 16])
def test_subseq_matches_oracle(kw, kind, d):
    rng = np.random.default_rng(100 + d + 10 * kind)
    limit = {1: 1024, 3: 512, 8: 256, 16: 128}[d]
    lengths = [1, 5, 31, 100, 128, 129, min(300, limit), limit]
    lengths = sorted(set(x for x in lengths if x <= limit))
    t = walk_series(rng, 3000, d)
    qs = []
    for m in lengths:
        a = int(rng.integers(0, 3000 - m))
        # a noisy, warped copy of a piece of T, so that a close match exists
        src = t[a:a + m + m // 4]
        idx = np.sort(rng.choice(len(src), size=m, replace=len(src) < m))
        qs.append((src[idx] + 0.05 * rng.standard_normal((m, d))).astype(np.float32))
    q = np.concatenate(qs)
    q_off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
    vals, ends = kw.subseq(cuda(q), cuda(q_off), cuda(t), distance=kind)
    vals, ends = vals.cpu().numpy(), ends.cpu().numpy()
    for i, x in enumerate(qs):
        check(kind, x, t, float(vals[i]), int(ends[i]))


@pytest.mark.parametrize("kind", [0, 1])
def test_subseq_eps_and_edges(kw, kind):
    rng = np.random.default_rng(5 + kind)
    d = 2
    t = walk_series(rng, 700, d)
    q = (t[200:260] + 0.1 * rng.standard_normal((60, d))).astype(np.float32)
    q_off = np.array([0, 60], dtype=np.int64)
    ov, oend = oracle.sub_distance(kind, q.astype(np.float64), t.astype(np.float64))
    for f, expect in ((2.0, True), (1.001, True), (0.5, False)):
        v, e = kw.subseq(q, q_off, t, distance=kind, eps=float(ov * f))
        if expect:
            assert float(v[0]) == pytest.approx(ov, rel=TOL[kind], abs=0) and int(e[0]) == oend
        else:
            assert math.isinf(float(v[0])) and int(e[0]) == -1
    # host inputs give the same as device inputs
    vh, eh = kw.subseq(q, q_off, t, distance=kind)
    vd, ed = kw.subseq(cuda(q), cuda(q_off), cuda(t), distance=kind)
    assert float(vh[0]) == float(vd.cpu()[0]) and int(eh[0]) == int(ed.cpu()[0])
    # an exact copy of the query inside T: 0 at the copy's end
    t2 = t.copy()
    t2[400:460] = q
    v, e = kw.subseq(q, q_off, t2, distance=kind)
    assert float(v[0]) == 0.0 and int(e[0]) == 459
    # series of one point, query of one point
    for tt, qq in ((t[:1], q), (t, q[:1]), (t[:1], q[:1])):
        qo = np.array([0, len(qq)], dtype=np.int64)
        v, e = kw.subseq(qq, qo, tt, distance=kind)
        check(kind, qq, tt, float(v[0]), int(e[0]))


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d,k", [(1, 5), (3, 16), (8, 2)])
def test_subseq_k_best_ends(kw, kind, d, k):
    """The k best ends against the oracle's: the same ends in the same order,
    values within the tolerance."""
    rng = np.random.default_rng(300 + 10 * d + kind)
    t = walk_series(rng, 2500, d)
    qs = []
    for m in (1, 17, 64, 150):
        a = int(rng.integers(0, 2500 - m))
        qs.append((t[a:a + m] + 0.05 * rng.standard_normal((m, d))).astype(np.float32))
    q = np.concatenate(qs)
    q_off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
    vals, ends = kw.subseq(cuda(q), cuda(q_off), cuda(t), distance=kind, k=k)
    vals, ends = vals.cpu().numpy(), ends.cpu().numpy()
    assert vals.shape == (len(qs), k)
    for i, x in enumerate(qs):
        ov, oe = oracle.sub_ends(kind, x.astype(np.float64), t.astype(np.float64), k)
        np.testing.assert_array_equal(ends[i], oe)
        np.testing.assert_allclose(vals[i], ov, rtol=TOL[kind], atol=0)
    # k = 1 of knn_subseq_k is knn_subseq
    v1, e1 = kw.subseq(cuda(q), cuda(q_off), cuda(t), distance=kind)
    np.testing.assert_array_equal(e1.cpu().numpy(), ends[:, 0])
    np.testing.assert_array_equal(v1.cpu().numpy(), vals[:, 0])
    with pytest.raises(kw.KnnError):
        kw.subseq(cuda(q), cuda(q_off), cuda(t), distance=kind, k=17)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d,stride", [(1, 1), (3, 3), (16, 2)])
def test_banded_subsequence_windows(kw, kind, d, stride):
    """Banded subsequence search: the k best length-m windows of T under the
    Sakoe-Chiba band, against the oracle's k-NN over the same windows written
    out explicitly (exact ids in order, distances within tolerance), and the
    eps form."""
    rng = np.random.default_rng(400 + d + stride + 10 * kind)
    n, m, k, band = 1500, 64, 6, 0.1
    t = walk_series(rng, n, d)
    qs = [(t[a:a + m] + 0.05 * rng.standard_normal((m, d))).astype(np.float32)
          for a in rng.integers(0, n - m, 4)]
    q = np.concatenate(qs)
    q_off = np.arange(len(qs) + 1, dtype=np.int64) * m
    starts = np.arange(0, n - m + 1, stride)
    win = np.concatenate([t[a:a + m] for a in starts])
    w_off = np.arange(len(starts) + 1, dtype=np.int64) * m
    db = kw.KnnDB.windows(cuda(t), m, stride)
    assert db.n == len(starts)
    ids, dist = db.scan(cuda(q), q_off, k=k, band=band, distance=kind)
    oids, odist = oracle.knn(win, w_off, q, q_off, band=float(np.float32(band)), kind=kind, k=k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_allclose(dist.cpu().numpy(), odist, rtol=TOL[kind], atol=0)
    eps = float(np.float32(odist[:, 3].max()))
    ei, ed, ec = db.scan(cuda(q), q_off, k=0, eps=eps, eps_capacity=len(starts), band=band,
                         distance=kind)
    oi, od, oc = oracle.knn(win, w_off, q, q_off, band=float(np.float32(band)), kind=kind, k=0,
                            eps=eps, cap=len(starts))
    np.testing.assert_array_equal(ec.cpu().numpy(), oc)
    for i in range(len(qs)):
        c = int(oc[i])
        assert set(ei.cpu().numpy()[i, :c].tolist()) == set(oi[i, :c].tolist())
    db.close()


def test_subseq_greedy_bound(kw):
    """Algorithm 2 on the GPU: an upper bound of the subsequence DK, equal to the
    oracle's walk except where FP32 breaks a near-tie differently."""
    rng = np.random.default_rng(11)
    d = 3
    t = walk_series(rng, 2000, d)
    qs = [(t[a:a + m] + 0.1 * rng.standard_normal((m, d))).astype(np.float32)
          for a, m in ((100, 40), (900, 200), (1200, 700), (10, 1))]
    q = np.concatenate(qs)
    q_off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
    ub, ue = kw.subseq(q, q_off, t, greedy=True)
    dk, _ = kw.subseq(q[: q_off[2]], q_off[:3], t, distance=1)   # the queries within 512
    same = 0
    for i, x in enumerate(qs):
        og, oe = oracle.sub_gdk(x.astype(np.float64), t.astype(np.float64))
        ov, _ = oracle.sub_distance(1, x.astype(np.float64), t.astype(np.float64))
        assert float(ub[i]) >= ov * (1 - 1e-6) - 1e-6
        if i < 2:
            assert float(ub[i]) >= float(dk[i]) * (1 - 1e-6)
        same += abs(float(ub[i]) - og) <= 1e-5 * max(og, 1.0) and int(ue[i]) == oe
    assert same >= 3
    # early exit below the bound
    v, e = kw.subseq(q[:40], q_off[:2], t, greedy=True, eps=float(ub[0]) * 0.5)
    assert float(v[0]) > float(ub[0]) * 0.5 and int(e[0]) == -1


def test_subseq_invalid(kw):
    t = np.zeros((100, 3), dtype=np.float32)
    q = np.zeros((600, 3), dtype=np.float32)
    with pytest.raises(kw.KnnError):
        kw.subseq(q, np.array([0, 600]), t)          # m above the d = 3 limit (512)
    with pytest.raises(kw.KnnError):
        kw.subseq(q[:10], np.array([0, 10]), t, distance=2)
    bad = t.copy()
    bad[5, 1] = np.nan
    with pytest.raises(kw.KnnError):
        kw.subseq(q[:10], np.array([0, 10]), bad)
    with pytest.raises(kw.KnnError):
        kw.subseq(q[:10], np.array([0, 10]), t, eps=-1.0)
    with pytest.raises(kw.KnnError):
        kw.subseq(q[:10], np.array([0, 0, 10]), t)   # an empty query
