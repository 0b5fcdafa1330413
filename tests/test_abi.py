"""The C-ABI library: it loads, exports every symbol include/knnwarp.h
declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "knnwarp.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"KNN_API\s+[\w\s\*]+?\b(knn_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def knnlib():
    import paper_1811_11076_gb300 as kw
    from paper_1811_11076_gb300 import build
    build.build()
    return kw.lib()


def test_header_declares_the_binding_exports():
    import paper_1811_11076_gb300 as kw
    assert declared_symbols() == sorted(kw.EXPORTS)


def test_library_exports_every_declared_symbol(knnlib):
    for name in declared_symbols():
        assert hasattr(knnlib, name), name


def test_status_strings(knnlib):
    assert knnlib.knn_status_string(0) == b"ok"
    assert knnlib.knn_status_string(1) == b"invalid argument"
    assert b"sm_103a" in knnlib.knn_version()


def test_null_arguments_rejected_before_any_launch(knnlib):
    out = C.c_void_p()
    assert knnlib.knn_db_create(None, None, 10, 3, None, C.byref(out)) == 1
    assert knnlib.knn_db_create(None, None, 10, 3, None, None) == 1
    assert knnlib.knn_db_destroy(None) == 1
    assert knnlib.knn_scan(None, None, None, 1, None, None, None, None, None, None) == 1
    assert b"NULL" in knnlib.knn_last_error()
