"""Parity at the benchmark's full size: d=3, 100,000 series of length 256,
1,000 queries scanned in one batch (the launch configuration bench.py times),
sampled queries checked one by one against the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_11076_gb300 as kw
    from paper_1811_11076_gb300 import build
    from synthdata import make_workload
    build.build()
    w = make_workload(n_series=100_000, n_queries=1000, d=3, length=256, n_classes=20, seed=1)
    db = kw.KnnDB(torch.from_numpy(w.db).cuda(), w.db_off)
    yield kw, w, db, torch.from_numpy(w.q).cuda()
    db.close()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("k,band,seed", [(10, 0.1, 3), (1, 0.05, 3), (10, 0.1, 0)])
def test_full_size_sampled(setup, kind, k, band, seed):
    kw, w, db, q = setup
    ids, dist = db.scan(q, w.q_off, k=k, band=band, distance=kind, seed=seed)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1000 * kind + k)
    sample = np.sort(rng.choice(1000, 4, replace=False))
    for qi in sample:
        qo = np.array([0, 256])
        oids, odist = oracle.knn(w.db, w.db_off, w.query(qi), qo, band=float(np.float32(band)),
                                 kind=kind, k=k, method=True, threads=os.cpu_count())
        assert list(ids[qi]) == list(oids[0]), (qi, ids[qi], oids[0])
        np.testing.assert_allclose(dist[qi], odist[0], rtol=1e-5 if kind == 0 else 1e-6)
    # properties that hold for every query: ascending, finite, distinct ids
    assert np.all(np.diff(dist, axis=1) >= 0)
    assert np.all(np.isfinite(dist))
    assert all(len(set(r)) == k for r in ids)
