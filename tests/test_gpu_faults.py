"""Failure paths, exercised without faulting the GPU.

Host side: KNN_FAULT_INJECT=alloc_after:N makes the library's N+1-th device
allocation fail; every entry point must return KNN_ERR_OOM, release what it
had allocated, and leave the database usable.  Device side:
KNN_FAULT_INJECT=wait makes the LB_Box launches (the coarse first stage or
the LB_Box stream, whichever runs) run one bounded wait on a
barrier that nothing completes (nothing is in flight on it); the wait gives
up after a short limit, the kernel reports it in the status word, and the
scan returns KNN_ERR_TIMEOUT.  The context stays usable in both cases.
"""
import numpy as np
import pytest

from synthdata import make_workload

pytestmark = pytest.mark.gpu

OOM, TIMEOUT = 2, 4


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


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failures_release_everything(kw, monkeypatch):
    import torch
    w = make_workload(n_series=3000, n_queries=6, d=3, length=64, n_classes=5, seed=3)
    dbx, q = torch.from_numpy(w.db).cuda(), torch.from_numpy(w.q).cuda()
    out = (torch.empty((6, 5), dtype=torch.int64, device="cuda"),
           torch.empty((6, 5), dtype=torch.float32, device="cuda"),
           torch.empty(6, dtype=torch.int64, device="cuda"))
    db = kw.KnnDB(dbx, w.db_off)
    db.scan(q, w.q_off, k=5, band=0.1, distance=kw.DTW, out=out)
    ref = (out[0].clone(), out[1].clone())
    assert torch.equal(out[0], ref[0])  # torch's own scratch for the comparison, before `base`
    db.close()
    base = _free()

    # knn_db_create fails at each of its allocations in turn
    failures = 0
    for n in range(64):
        monkeypatch.setenv("KNN_FAULT_INJECT", f"alloc_after:{n}")
        try:
            db = kw.KnnDB(dbx, w.db_off)
        except kw.KnnError as e:
            monkeypatch.delenv("KNN_FAULT_INJECT")
            assert e.status == OOM
            assert _free() == base, f"allocation {n}: device memory not released"
            failures += 1
            continue
        monkeypatch.delenv("KNN_FAULT_INJECT")
        db.close()
        break
    assert failures >= 3 and _free() == base

    # knn_scan fails at each allocation of its workspace in turn (a fresh
    # database each time, so that every workspace buffer is allocated
    # again); each failure leaves the database usable, and closing it returns
    # every byte
    failures = 0
    for n in range(64):
        db = kw.KnnDB(dbx, w.db_off)
        monkeypatch.setenv("KNN_FAULT_INJECT", f"alloc_after:{n}")
        try:
            db.scan(q, w.q_off, k=5, band=0.1, distance=kw.DTW, out=out)
            failed = False
        except kw.KnnError as e:
            assert e.status == OOM
            failed = True
        monkeypatch.delenv("KNN_FAULT_INJECT")
        db.scan(q, w.q_off, k=5, band=0.1, distance=kw.DTW, out=out)
        assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
        db.close()
        assert _free() == base, f"scan allocation {n}: device memory not released"
        if not failed:
            break
        failures += 1
    assert failures >= 3


def test_device_wait_gives_up_and_reports_timeout(kw, monkeypatch):
    import torch
    w = make_workload(n_series=2000, n_queries=8, d=3, length=64, n_classes=5, seed=4)
    db = kw.KnnDB(torch.from_numpy(w.db).cuda(), w.db_off)
    q = torch.from_numpy(w.q).cuda()
    for kind in (kw.DTW, kw.DK):
        ref = db.scan(q, w.q_off, k=4, band=0.1, distance=kind)
        monkeypatch.setenv("KNN_FAULT_INJECT", "wait")
        with pytest.raises(kw.KnnError) as e:
            db.scan(q, w.q_off, k=4, band=0.1, distance=kind)
        monkeypatch.delenv("KNN_FAULT_INJECT")
        assert e.value.status == TIMEOUT
        again = db.scan(q, w.q_off, k=4, band=0.1, distance=kind)
        assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])
    db.close()
