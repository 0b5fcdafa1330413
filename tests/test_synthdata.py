"""The seeded input generators: reproducible, prefix-consistent, recipe shapes."""
import numpy as np

from synthdata import make_long_series, make_workload


def test_database_prefix_and_queries_do_not_depend_on_size():
    a = make_workload(n_series=3000, n_queries=7, d=4, length=40, n_classes=6, seed=3)
    b = make_workload(n_series=1500, n_queries=7, d=4, length=40, n_classes=6, seed=3)
    assert np.array_equal(b.db, a.db[: b.db_off[-1]])
    assert np.array_equal(b.db_labels, a.db_labels[:1500])
    assert np.array_equal(b.q, a.q) and np.array_equal(b.q_labels, a.q_labels)
    c = make_workload(n_series=3000, n_queries=7, d=4, length=40, n_classes=6, seed=3, threads=1)
    assert np.array_equal(c.db, a.db) and np.array_equal(c.q, a.q)


def test_uneven_lengths_and_layout():
    w = make_workload(n_series=2500, n_queries=5, d=3, length_range=(50, 90), n_classes=4, seed=1)
    lens = np.diff(w.db_off)
    assert lens.min() >= 50 and lens.max() <= 90 and len(np.unique(lens)) > 30
    assert w.db.dtype == np.float32 and w.db.shape == (int(w.db_off[-1]), 3)
    assert np.all(np.isfinite(w.db)) and np.all(np.isfinite(w.q))
    q2 = make_workload(n_series=10, n_queries=5, d=3, length_range=(50, 90), n_classes=4, seed=1)
    assert np.array_equal(q2.q_off, w.q_off) and np.array_equal(q2.q, w.q)


def test_instances_follow_their_class_template():
    # noise sigma 0.1 around a warped template: a series is much closer (in
    # the mean over points of the nearest template value) to its own class
    w = make_workload(n_series=200, n_queries=0, d=2, length=64, n_classes=3, seed=9,
                      noise_sigma=0.0)
    same, other = [], []
    for i in range(0, 200, 7):
        for j in range(1, 200, 11):
            x, y = w.series(i), w.series(j)
            dist = float(np.mean(np.min(np.sum((x[:, None] - y[None]) ** 2, axis=2), axis=1)))
            (same if w.db_labels[i] == w.db_labels[j] else other).append(dist)
    assert np.median(same) < 0.1 * np.median(other)


def test_long_series_shapes_and_reproducibility():
    L = make_long_series(n=20000, n_queries=3, d=2, q_length=64, seed=2)
    assert L.t.shape == (20000, 2) and L.q.shape == (3 * 64, 2)
    assert np.array_equal(L.q_off, np.arange(4) * 64)
    M = make_long_series(n=20000, n_queries=3, d=2, q_length=64, seed=2)
    assert np.array_equal(L.t, M.t) and np.array_equal(L.q, M.q)
