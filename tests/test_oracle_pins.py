"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics.

None of these re-types the oracle's own dynamic program.  The pins are
brute-force enumeration of warping paths, closed forms, the inequalities the
paper proves (Section 3, Eq. 1; Section 4.1), SciPy's sliding-window filters
for the envelope, and the paper's own LB_Box failure example (Figure 2).
"""
import itertools
import math

import numpy as np
import pytest
from scipy.ndimage import maximum_filter1d, minimum_filter1d

INF = float("inf")


# ---------------------------------------------------------------------------
# brute force: enumerate every warping path explicitly

def all_paths(m, n, r):
    """Every monotone path (0,0)->(m-1,n-1) with unit steps inside |i-j|<=r."""
    out = []

    def rec(i, j, acc):
        if abs(i - j) > r:
            return
        acc = acc + [(i, j)]
        if i == m - 1 and j == n - 1:
            out.append(acc)
            return
        if i + 1 < m:
            rec(i + 1, j, acc)
        if j + 1 < n:
            rec(i, j + 1, acc)
        if i + 1 < m and j + 1 < n:
            rec(i + 1, j + 1, acc)

    rec(0, 0, [])
    return out


def brute_dtw(s, t, r):
    paths = all_paths(len(s), len(t), r)
    if not paths:
        return INF
    return min(sum(float(np.sum((s[i] - t[j]) ** 2)) for i, j in p) for p in paths)


def brute_dk(s, t, r):
    paths = all_paths(len(s), len(t), r)
    if not paths:
        return INF
    return min(max(math.sqrt(float(np.sum((s[i] - t[j]) ** 2))) for i, j in p) for p in paths)


def rand_series(rng, n, d):
    return rng.standard_normal((n, d))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dp_matches_path_enumeration(orc, d):
    rng = np.random.default_rng(100 + d)
    for trial in range(40):
        m = int(rng.integers(1, 7))
        n = int(rng.integers(1, 7))
        r = int(rng.choice([0, 1, 2, 3, 10]))
        s = rand_series(rng, m, d)
        t = rand_series(rng, n, d)
        bd, bk = brute_dtw(s, t, r), brute_dk(s, t, r)
        od, ok = orc.dtw(s, t, r), orc.dk(s, t, r)
        if bd == INF:
            assert od == INF and ok == INF
            continue
        assert od == pytest.approx(bd, rel=1e-12, abs=1e-12)
        assert ok == pytest.approx(bk, rel=1e-12, abs=1e-12)


def test_unreachable_end_is_inf(orc):
    s = np.zeros((3, 2))
    t = np.zeros((7, 2))
    assert orc.dtw(s, t, 3) == INF          # |m-n| = 4 > r
    assert orc.dk(s, t, 3) == INF
    assert orc.dtw(s, t, 4) == 0.0


# ---------------------------------------------------------------------------
# closed forms

def test_zero_band_is_lockstep(orc):
    rng = np.random.default_rng(1)
    s, t = rand_series(rng, 9, 3), rand_series(rng, 9, 3)
    c = np.sum((s - t) ** 2, axis=1)
    assert orc.dtw(s, t, 0) == pytest.approx(c.sum(), rel=1e-13)
    assert orc.dk(s, t, 0) == pytest.approx(np.sqrt(c).max(), rel=1e-13)


def test_constant_series(orc):
    a = np.array([1.0, -2.0, 0.5])
    b = np.array([0.0, 1.0, 2.5])
    s = np.tile(a, (5, 1))
    t = np.tile(b, (8, 1))
    sq = float(np.sum((a - b) ** 2))
    assert orc.dtw(s, t, 8) == pytest.approx(8 * sq, rel=1e-13)
    assert orc.dk(s, t, 8) == pytest.approx(math.sqrt(sq), rel=1e-13)


def test_identity_and_symmetry(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        m, n = int(rng.integers(2, 30)), int(rng.integers(2, 30))
        r = int(rng.integers(abs(m - n), 30))
        s, t = rand_series(rng, m, 2), rand_series(rng, n, 2)
        assert orc.dtw(s, s, r) == 0.0 and orc.dk(s, s, r) == 0.0
        assert orc.dtw(s, t, r) == pytest.approx(orc.dtw(t, s, r), rel=1e-12)
        assert orc.dk(s, t, r) == orc.dk(t, s, r)


def test_dk_squared_below_dtw_and_endpoints(orc):
    rng = np.random.default_rng(3)
    for _ in range(30):
        m, n = int(rng.integers(2, 40)), int(rng.integers(2, 40))
        r = int(rng.integers(abs(m - n), 40))
        s, t = rand_series(rng, m, 3), rand_series(rng, n, 3)
        dtw, dk = orc.dtw(s, t, r), orc.dk(s, t, r)
        assert dk * dk <= dtw * (1 + 1e-12)
        # every path starts at (0,0) and ends at (m-1,n-1)
        assert dk >= np.linalg.norm(s[0] - t[0]) - 1e-12
        assert dk >= np.linalg.norm(s[-1] - t[-1]) - 1e-12


def test_monotone_in_band(orc):
    rng = np.random.default_rng(4)
    s, t = rand_series(rng, 30, 2), rand_series(rng, 30, 2)
    prev_dtw, prev_dk = INF, INF
    for r in range(0, 31):
        d1, d2 = orc.dtw(s, t, r), orc.dk(s, t, r)
        assert d1 <= prev_dtw * (1 + 1e-12) and d2 <= prev_dk
        prev_dtw, prev_dk = d1, d2


def test_band_radius_rule(orc):
    assert orc.band_radius(256, 256, 0.05) == 12
    assert orc.band_radius(256, 256, 0.10) == 25
    assert orc.band_radius(64, 64, 0.10) == 6
    assert orc.band_radius(100, 300, 0.10) == 30
    assert orc.band_radius(5, 9, 1.0) == 9


# ---------------------------------------------------------------------------
# envelope and lower bounds (Sections 2.3 and 3)

def scipy_envelope(t, r, length):
    """Clipped-window min/max via SciPy; 'nearest' padding repeats edge values,
    which never changes a window's min or max."""
    n = t.shape[0]
    lo = minimum_filter1d(t, size=2 * r + 1, axis=0, mode="nearest")
    hi = maximum_filter1d(t, size=2 * r + 1, axis=0, mode="nearest")
    L = np.full((length, t.shape[1]), np.inf)
    U = np.full((length, t.shape[1]), -np.inf)
    k = min(length, n)
    L[:k], U[:k] = lo[:k], hi[:k]
    for i in range(n, length):          # windows reaching past the end
        a = max(0, i - r)
        if a <= n - 1:
            L[i], U[i] = t[a:].min(axis=0), t[a:].max(axis=0)
    return L, U


def test_envelope_matches_scipy(orc):
    rng = np.random.default_rng(5)
    for r in [0, 1, 3, 12]:
        t = rand_series(rng, 50, 3)
        for length in [50, 57]:
            lo, hi = orc.envelope(t, r, length)
            L, U = scipy_envelope(t, r, length)
            np.testing.assert_array_equal(lo, L)
            np.testing.assert_array_equal(hi, U)


def keogh_1d_textbook(s, t, r):
    """LB_Keogh as in Section 2.3, with the envelope from SciPy."""
    lo = minimum_filter1d(t, size=2 * r + 1, mode="nearest")[: len(s)]
    hi = maximum_filter1d(t, size=2 * r + 1, mode="nearest")[: len(s)]
    e = np.where(s < lo, lo - s, np.where(s > hi, s - hi, 0.0))
    return float(np.sum(e * e))


def test_lb_box_is_sum_of_per_dimension_keogh(orc):
    """Eq. 1: LB_Box(S,T) = sum_j LB_Keogh(S^j, T^j); and LB_Box == LB_Keogh at d=1."""
    rng = np.random.default_rng(6)
    for d in [1, 2, 3, 5]:
        for r in [0, 2, 7]:
            s, t = rand_series(rng, 40, d), rand_series(rng, 40, d)
            per_dim = sum(keogh_1d_textbook(s[:, j], t[:, j], r) for j in range(d))
            assert orc.lb_box(s, t, r) == pytest.approx(per_dim, rel=1e-12, abs=1e-12)
            if d == 1:
                assert orc.lb_box(s, t, r) == pytest.approx(orc.lb_keogh_1d(s, t, r), rel=1e-14)
                assert orc.lb_keogh_1d(s, t, r) == pytest.approx(
                    keogh_1d_textbook(s[:, 0], t[:, 0], r), rel=1e-12, abs=1e-12)


def test_lower_bound_chain(orc):
    """Section 3: LB_Box <= LB_Sigma-min <= DTW; and the max form bounds DK^2."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        d = int(rng.integers(1, 6))
        m = int(rng.integers(5, 40))
        n = int(np.clip(m + rng.integers(-4, 5), 2, None))
        r = int(rng.integers(abs(m - n), 12))
        s, t = rand_series(rng, m, d), rand_series(rng, n, d)
        box, smin, dtw = orc.lb_box(s, t, r), orc.lb_sigma_min(s, t, r), orc.dtw(s, t, r)
        assert box <= smin * (1 + 1e-12) + 1e-12
        assert smin <= dtw * (1 + 1e-12) + 1e-12
        dk = orc.dk(s, t, r)
        assert orc.lb_box(s, t, r, form=1) <= dk * dk * (1 + 1e-12) + 1e-12
        # the envelope may sit on either side: banded DTW is symmetric
        assert orc.lb_box(t, s, r) <= dtw * (1 + 1e-12) + 1e-12


def test_lb_box_brute_small(orc):
    """LB_Box against the definition min_{t in B_i} ||s_i - t||^2, brute-forced on a grid."""
    rng = np.random.default_rng(8)
    s, t = rand_series(rng, 6, 2), rand_series(rng, 6, 2)
    r = 1
    per_point = []
    for i in range(6):
        w = t[max(0, i - r): i + r + 1]
        lo, hi = w.min(axis=0), w.max(axis=0)
        gx = np.linspace(lo[0], hi[0], 401)
        gy = np.linspace(lo[1], hi[1], 401)
        X, Y = np.meshgrid(gx, gy)
        per_point.append(float(np.min((X - s[i, 0]) ** 2 + (Y - s[i, 1]) ** 2)))
    total, worst = sum(per_point), max(per_point)
    # the grid minimum can only overshoot the true minimum, by O(spacing^2)
    lb = orc.lb_box(s, t, r)
    assert lb <= total + 1e-12 and total - lb < 1e-4 * (1.0 + total)
    # the max form: the largest per-point box distance (the DK^2 bound)
    lbm = orc.lb_box(s, t, r, form=1)
    assert lbm <= worst + 1e-12 and worst - lbm < 1e-4 * (1.0 + worst)


def test_segment_box_bound(orc):
    """The cascade's coarse stage: with W = 1 it is LB_Box itself (each
    segment one point, its box B_i); for every W it never exceeds LB_Box (in
    either form); hand-worked values."""
    import json
    import os
    rng = np.random.default_rng(21)
    for _ in range(60):
        d = int(rng.integers(1, 5))
        m = int(rng.integers(4, 40))
        n = int(np.clip(m + rng.integers(-3, 4), 2, None))
        r = int(rng.integers(abs(m - n), 10))
        s, t = rand_series(rng, m, d), rand_series(rng, n, d)
        for form in (0, 1):
            box = orc.lb_box(s, t, r, form=form)
            assert orc.lb_seg(s, t, r, 1, form) == pytest.approx(box, rel=1e-12, abs=1e-12)
            for W in (2, 4, 16):
                assert orc.lb_seg(s, t, r, W, form) <= box * (1 + 1e-12) + 1e-12
    # the 64-point segments used for wide points on series of >= 256 points
    positive = 0
    for _ in range(6):
        d = int(rng.integers(8, 17))
        m = int(rng.integers(256, 320))
        n = int(np.clip(m + rng.integers(-5, 6), 256, None))
        r = int(rng.integers(abs(m - n), 30))
        # smooth walks (on iid noise a 64-point mean sits inside its box)
        s = np.cumsum(rand_series(rng, m, d), axis=0)
        t = np.cumsum(rand_series(rng, n, d), axis=0) + 3.0
        for form in (0, 1):
            box = orc.lb_box(s, t, r, form=form)
            seg = orc.lb_seg(s, t, r, 64, form)
            assert seg <= box * (1 + 1e-12) + 1e-12
            positive += seg > 0
    assert positive > 0
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")) as f:
        cases = json.load(f)["segment_box_cases"]
    for c in cases:
        s, t = np.array(c["S"], dtype=float), np.array(c["T"], dtype=float)
        assert orc.lb_seg(s, t, c["r"], c["W"], 0) == pytest.approx(c["lb_seg"], rel=1e-12), c["name"]
        assert orc.lb_seg(s, t, c["r"], c["W"], 1) == pytest.approx(c["lb_seg_max"], rel=1e-12)
        assert orc.lb_box(s, t, c["r"]) == pytest.approx(c["lb_box"], rel=1e-12), c["name"]


# ---------------------------------------------------------------------------
# Section 4: GDK, sparse DK, early abandoning

def test_gdk_is_an_upper_bound_and_a_path_value(orc):
    rng = np.random.default_rng(9)
    for _ in range(60):
        d = int(rng.integers(1, 4))
        m, n = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        r = int(rng.choice([1, 2, 6]))
        s, t = rand_series(rng, m, d), rand_series(rng, n, d)
        g, gs = orc.gdk(s, t, r), orc.greedy_dtw(s, t, r)
        dk, dtw = orc.dk(s, t, r), orc.dtw(s, t, r)
        if dk == INF:
            assert g == INF
            continue
        assert g >= dk - 1e-12 and gs >= dtw - 1e-12
        # both greedy values belong to ONE admissible path: its max of Euclidean
        # costs is GDK and its sum of squared costs is the DTW greedy bound
        paths = all_paths(m, n, r)
        pairs = {(round(max(math.sqrt(float(np.sum((s[i] - t[j]) ** 2))) for i, j in p), 10),
                  round(sum(float(np.sum((s[i] - t[j]) ** 2)) for i, j in p), 10))
                 for p in paths}
        assert (round(g, 10), round(gs, 10)) in pairs


def test_gdk_zero_band_equals_dk(orc):
    rng = np.random.default_rng(10)
    s, t = rand_series(rng, 12, 3), rand_series(rng, 12, 3)
    assert orc.gdk(s, t, 0) == pytest.approx(orc.dk(s, t, 0), rel=1e-14)


def test_gdk_threshold_returns_early(orc):
    rng = np.random.default_rng(11)
    s, t = rand_series(rng, 20, 2), rand_series(rng, 20, 2)
    full = orc.gdk(s, t, 5)
    early = orc.gdk(s, t, 5, eps=full * 0.5)
    assert early > full * 0.5


def test_sparse_dk(orc):
    rng = np.random.default_rng(12)
    for _ in range(60):
        d = int(rng.integers(1, 4))
        m = int(rng.integers(1, 25))
        n = int(np.clip(m + rng.integers(-3, 4), 1, None))
        r = int(rng.integers(abs(m - n), 25))
        s, t = rand_series(rng, m, d), rand_series(rng, n, d)
        dk = orc.dk(s, t, r)
        v, _ = orc.sparse_dk(s, t, r, INF)
        assert v == dk
        if dk == INF:
            continue
        for eps in [dk, dk * 1.5, dk * 0.999, dk * 0.5]:
            v, cells = orc.sparse_dk(s, t, r, eps)
            assert v == (dk if dk <= eps else INF)


def test_sparse_dk_visits_few_cells_under_tight_threshold(orc):
    rng = np.random.default_rng(13)
    s = np.cumsum(rng.standard_normal((200, 3)), axis=0)
    t = s + 0.01 * rng.standard_normal((200, 3))
    far = s + 50.0
    dk = orc.dk(s, t, 20)
    _, cells_near = orc.sparse_dk(s, t, 20, dk)
    _, cells_far = orc.sparse_dk(s, far, 20, dk)
    assert cells_far <= 2 and cells_near < 200 * 41


def test_dtw_abandon(orc):
    rng = np.random.default_rng(14)
    for _ in range(40):
        m = int(rng.integers(1, 30))
        n = int(np.clip(m + rng.integers(-3, 4), 1, None))
        r = int(rng.integers(abs(m - n), 30))
        s, t = rand_series(rng, m, 2), rand_series(rng, n, 2)
        dtw = orc.dtw(s, t, r)
        for eps in [INF, dtw, dtw * 0.9]:
            v, _ = orc.dtw_abandon(s, t, r, eps)
            assert v == (dtw if dtw <= eps else INF)


# ---------------------------------------------------------------------------
# The paper's LB_Box failure case (Section 3, Figure 2): T runs along the left
# and then the bottom edge of its bounding box while the query point sits on
# the top-right corner; LB_Box sees zero, LB_Sigma-min does not.

def test_figure2_example(orc):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "figure2_box.json")) as f:
        g = json.load(f)
    s = np.array(g["S"], dtype=float)
    t = np.array(g["T"], dtype=float)
    r = g["r"]
    assert orc.lb_box(s, t, r) == pytest.approx(g["lb_box"], abs=1e-12)
    assert orc.lb_sigma_min(s, t, r) == pytest.approx(g["lb_sigma_min"], rel=1e-12)
    assert orc.dtw(s, t, r) == pytest.approx(g["dtw"], rel=1e-12)
    assert orc.dk(s, t, r) == pytest.approx(g["dk"], rel=1e-12)


def test_hand_computed_examples(orc):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        s = np.array(c["S"], dtype=float)
        t = np.array(c["T"], dtype=float)
        assert orc.dtw(s, t, c["r"]) == pytest.approx(c["dtw"], rel=1e-12), c["name"]
        assert orc.dk(s, t, c["r"]) == pytest.approx(c["dk"], rel=1e-12), c["name"]
        if "gdk" in c:
            assert orc.gdk(s, t, c["r"]) == pytest.approx(c["gdk"], rel=1e-12), c["name"]
        if "lb_box" in c:
            assert orc.lb_box(s, t, c["r"]) == pytest.approx(c["lb_box"], rel=1e-12,
                                                             abs=1e-12), c["name"]
        if "lb_box_max" in c:
            assert orc.lb_box(s, t, c["r"], form=1) == pytest.approx(
                c["lb_box_max"], rel=1e-12, abs=1e-12), c["name"]
        if "greedy_dtw" in c:
            assert orc.greedy_dtw(s, t, c["r"]) == pytest.approx(
                c["greedy_dtw"], rel=1e-12), c["name"]


# ---------------------------------------------------------------------------
# k-NN / eps-NN: the pruned method equals the plain definition

def _small_workload(d=2, N=300, L=32, Q=6, seed=0, length_range=None):
    from synthdata import make_workload
    return make_workload(n_series=N, n_queries=Q, d=d, length=L, n_classes=5, seed=seed,
                         length_range=length_range)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("k", [1, 5])
def test_knn_method_equals_plain(orc, kind, k):
    w = _small_workload()
    a = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=k)
    b = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=k, method=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("kind", [0, 1])
def test_knn_uneven_lengths_method_equals_plain(orc, kind):
    w = _small_workload(N=200, length_range=(20, 40), seed=3)
    a = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=3)
    b = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=3, method=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_knn_plain_is_sorted_definition(orc):
    w = _small_workload(N=120, Q=3)
    ids, dist = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=0, k=7)
    for qi in range(3):
        q = w.query(qi)
        r = orc.band_radius(len(q), 32, 0.1)
        all_d = [orc.dtw(q, w.series(c), r) for c in range(120)]
        order = sorted(range(120), key=lambda c: (all_d[c], c))[:7]
        assert list(ids[qi]) == order


@pytest.mark.parametrize("kind", [0, 1])
def test_eps_nn(orc, kind):
    w = _small_workload(N=200)
    ids, dist = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=20)
    eps = float(np.median(dist[:, 10]))
    a = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=0, eps=eps, cap=50)
    b = orc.knn(w.db, w.db_off, w.q, w.q_off, band=0.1, kind=kind, k=0, eps=eps, cap=50,
                method=True)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    for qi in range(w.n_queries):
        c = a[2][qi]
        assert np.all(a[1][qi, :min(c, 50)] <= eps)
        # consistent with k-NN: the eps ball is a prefix of the k-NN list
        inside = dist[qi] <= eps
        np.testing.assert_array_equal(a[0][qi, :inside.sum()], ids[qi][inside])


def test_knn_ties_broken_by_id(orc):
    w = _small_workload(N=50, Q=2)
    db = np.concatenate([w.db, w.db[:32], w.db[:32]])          # series 0 duplicated twice
    off = np.concatenate([w.db_off, w.db_off[-1] + np.array([32, 64])])
    q = w.db[:32].copy()
    ids, dist = orc.knn(db, off, q, np.array([0, 32]), band=0.1, kind=0, k=3, method=True)
    assert list(ids[0]) == [0, 50, 51] and dist[0, 0] == 0.0 == dist[0, 2]


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("band", [0.2, 0.5, 1.0])
def test_pairwise_matches_path_enumeration(orc, kind, band):
    """The pair list form (knn_pairwise's oracle): each listed pair of two
    different sets of uneven series against brute force over all warping
    paths, including pairs whose end cell lies outside the band (+inf)."""
    rng = np.random.default_rng(int(band * 10) + 7 * kind)
    la, lb_ = [1, 3, 4, 6, 5], [2, 6, 1, 5]
    a = [rand_series(rng, n, 2) for n in la]
    b = [rand_series(rng, n, 2) for n in lb_]
    a_off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb_)]).astype(np.int64)
    pairs = [(i, j) for i in range(len(a)) for j in range(len(b))]
    order = rng.permutation(len(pairs))
    pa = np.array([pairs[o][0] for o in order] + [2, 2])
    pb = np.array([pairs[o][1] for o in order] + [1, 1])
    bf = float(np.float32(band))
    got = orc.pairwise(np.concatenate(a), a_off, np.concatenate(b), b_off, pa, pb, band=bf,
                       kind=kind)
    brute = brute_dtw if kind == 0 else brute_dk
    n_inf = 0
    for x, (i, j) in enumerate(zip(pa, pb)):
        r = orc.band_radius(la[i], lb_[j], bf)
        exp = brute(a[i], b[j], r)
        n_inf += exp == INF
        assert got[x] == pytest.approx(exp, rel=1e-12, abs=1e-12), (i, j, r)
    assert (n_inf > 0) == (band < 1.0)


# --- subsequence search (Algorithm 2; Algorithm 3 with SUB = true) ----------

import oracle  # noqa: E402  (the same module the orc fixture provides)

def _brute_sub(kind, s, t):
    """min over every subsequence T[a..b] of the whole-match distance (no band),
    and for each end b the best value over starts a."""
    m, n = len(s), len(t)
    per_end = []
    for b in range(n):
        best_b = math.inf
        for a in range(b + 1):
            seg = t[a:b + 1]
            r = max(m, len(seg))
            v = oracle.dtw(s, seg, r) if kind == 0 else oracle.dk(s, seg, r)
            best_b = min(best_b, v)
        per_end.append(best_b)
    return min(per_end), per_end


@pytest.mark.parametrize("kind", [0, 1])
def test_subsequence_equals_min_over_all_subsequences(kind):
    """The free-start/free-end DP equals the minimum, over every subsequence of
    T, of the whole-match distance (itself pinned by path enumeration), and its
    end column is an end at which that minimum is attained."""
    rng = np.random.default_rng(7)
    for trial in range(40):
        d = int(rng.integers(1, 4))
        m = int(rng.integers(1, 5))
        n = int(rng.integers(1, 10))
        s = rng.standard_normal((m, d))
        t = rng.standard_normal((n, d))
        v, end = oracle.sub_distance(kind, s, t)
        bv, per_end = _brute_sub(kind, s, t)
        assert math.isclose(v, bv, rel_tol=1e-12, abs_tol=1e-12), (trial, v, bv)
        assert 0 <= end < n and math.isclose(per_end[end], bv, rel_tol=1e-12, abs_tol=1e-12)
        # the smallest such end
        assert all(per_end[b] > bv * (1 + 1e-12) + 1e-12 for b in range(end))


@pytest.mark.parametrize("kind", [0, 1])
def test_subsequence_k_best_ends(kind):
    """The k best ends: the per-end values of the brute force over every
    subsequence, k smallest by (value, end); k = 1 is sub_distance's answer."""
    rng = np.random.default_rng(17)
    for trial in range(30):
        d = int(rng.integers(1, 4))
        m = int(rng.integers(1, 5))
        n = int(rng.integers(1, 10))
        s = rng.standard_normal((m, d))
        t = rng.standard_normal((n, d))
        _, per_end = _brute_sub(kind, s, t)
        k = int(rng.integers(1, n + 3))
        vals, ends = oracle.sub_ends(kind, s, t, k)
        expect = sorted((per_end[b], b) for b in range(n))[:k]
        for j, (ev, eb) in enumerate(expect):
            assert math.isclose(vals[j], ev, rel_tol=1e-12, abs_tol=1e-12) and ends[j] == eb
        assert all(ends[j] == -1 and math.isinf(vals[j]) for j in range(len(expect), k))
        v1, e1 = oracle.sub_distance(kind, s, t)
        assert math.isclose(vals[0], v1, rel_tol=1e-12, abs_tol=1e-12) and ends[0] == e1


def test_subsequence_sparse_dk_matches_plain_within_eps():
    """Algorithm 3 with SUB = true visits only cells of cost <= eps: it returns
    the subsequence DK when that is <= eps and +inf otherwise, never another
    value, and visits fewer cells for a tighter eps."""
    rng = np.random.default_rng(8)
    for trial in range(60):
        d = int(rng.integers(1, 4))
        m = int(rng.integers(1, 7))
        n = int(rng.integers(1, 30))
        s = rng.standard_normal((m, d))
        t = rng.standard_normal((n, d))
        v, end = oracle.sub_distance(1, s, t)
        last_cells = None
        for f in (4.0, 2.0, 1.0 + 1e-9, 0.999, 0.5):
            sv, send, cells = oracle.sub_sparse_dk(s, t, v * f)
            if v <= v * f:
                assert sv == pytest.approx(v, rel=1e-12) and send == end
            else:
                assert sv == math.inf and send == -1
            if last_cells is not None:
                assert cells <= last_cells
            last_cells = cells
        assert oracle.sub_sparse_dk(s, t, math.inf)[0] == pytest.approx(v, rel=1e-12)


def test_subsequence_greedy_bounds_and_exact_copy():
    """Algorithm 2 walks one admissible path, so it bounds the subsequence DK
    from above; an exact copy of S inside T gives 0 for both, ending where the
    copy ends."""
    rng = np.random.default_rng(9)
    for trial in range(60):
        d = int(rng.integers(1, 4))
        m = int(rng.integers(1, 7))
        n = int(rng.integers(1, 30))
        s = rng.standard_normal((m, d))
        t = rng.standard_normal((n, d))
        v, _ = oracle.sub_distance(1, s, t)
        g, gend = oracle.sub_gdk(s, t)
        assert g >= v - 1e-12
        assert 0 <= gend < n
        # early exit: a threshold below the bound returns a value above it
        if g > 0:
            ge, _ = oracle.sub_gdk(s, t, 0.5 * g)
            assert ge > 0.5 * g
    s = rng.standard_normal((5, 2))
    t = rng.standard_normal((40, 2))
    t[17:22] = s
    for kind in (0, 1):
        v, end = oracle.sub_distance(kind, s, t)
        assert v == 0.0 and end == 21
    g, gend = oracle.sub_gdk(s, t)
    assert g == 0.0 and gend == 21
