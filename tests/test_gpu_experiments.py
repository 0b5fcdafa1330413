"""The LB_Box tightness sweep and the 1-NN accuracy experiment (bench.py
--experiment): their GPU statistics equal the oracle's on a small grid."""
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


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


@pytest.mark.parametrize("data", ["iid", "classes"])
def test_tightness_matches_oracle(kw, bench, data):
    band = 0.1
    rows = bench.tightness_table(kw, (1, 4), (16, 40), 24, band, data, seed=3)
    rng = np.random.default_rng(3)
    from synthdata import make_workload
    for row in rows:
        d, n = row["d"], row["n"]
        # the same draws as the table (same generator calls in the same order)
        if data == "iid":
            S = rng.random((24, n, d), dtype=np.float32)
            T = rng.random((24, n, d), dtype=np.float32)
        else:
            w = make_workload(n_series=48, n_queries=1, d=d, length=n, n_classes=10,
                              seed=3 + d * 1000 + n)
            X = w.db.reshape(48, n, d)
            S, T = X[:24], X[24:]
        r = oracle.band_radius(n, n, float(np.float32(band)))
        lb = np.array([oracle.lb_box(T[i], S[i], r) for i in range(24)])
        dtw = np.array([oracle.dtw(S[i], T[i], r) for i in range(24)])
        ok = dtw > 0
        assert row["mean_ratio"] == pytest.approx(float(np.mean(lb[ok] / dtw[ok])), rel=1e-4)
        assert row["ratio_of_means"] == pytest.approx(float(lb.mean() / dtw.mean()), rel=1e-4)
        assert 0.0 <= row["mean_ratio"] <= 1.0


def test_accuracy_matches_oracle(kw, bench):
    band = 0.1
    rows = bench.accuracy_table(kw, (2, 5), (32,), 300, 24, band, seed=4, noise=2.0)
    from synthdata import make_workload
    for row in rows:
        d, n = row["d"], row["n"]
        w = make_workload(n_series=300, n_queries=24, d=d, length=n, n_classes=10,
                          seed=4 + d * 1000 + n, noise_sigma=2.0)
        for kind, name in ((0, "dtw"), (1, "dk")):
            oids, _ = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=float(np.float32(band)),
                                 kind=kind, k=1)
            assert row["ids_" + name] == list(oids[:, 0])
            acc = float(np.mean(w.db_labels[oids[:, 0]] == w.q_labels))
            assert row["acc_" + name] == pytest.approx(acc)
