"""The C ABI library builds, loads and exports every symbol include/mecuco.h
declares (no compute calls: this runs on the CPU-only host too)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "mecuco.h")).read()
    return sorted(set(re.findall(r"MECUCO_API\s+[\w\s\*]+?\b(mecuco_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_06329_gb300 import build, _native
    build.build()
    return _native.load()


def test_header_declares_the_entry_points():
    names = _declared_functions()
    assert {"mecuco_create", "mecuco_destroy", "mecuco_knn", "mecuco_curvature",
            "mecuco_curvature_host", "mecuco_get_last_status", "mecuco_status_string"} <= set(names)


def test_library_exports_every_declared_symbol(lib):
    from paper_2606_06329_gb300 import _native
    names = _declared_functions()
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
    # the Python binding declares exactly the header's functions
    assert sorted(_native.SIGNATURES) == names


def test_status_strings(lib):
    from paper_2606_06329_gb300 import _native as N
    for code in range(7):
        s = lib.mecuco_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.mecuco_status_string(99).decode() == "unknown status"
    assert lib.mecuco_status_string(N.OK).decode() == "ok"


def test_argument_errors_need_no_gpu(lib):
    from paper_2606_06329_gb300 import _native as N
    # NULL handle / NULL output are rejected before any CUDA call
    assert lib.mecuco_create(None, 0) == N.ERR_INVALID_ARG
    assert lib.mecuco_destroy(None) == N.OK
    assert lib.mecuco_set_option(None, 0, 1) == N.ERR_INVALID_ARG
    assert lib.mecuco_knn(None, None, 0, 10, 4, 4, 3, 0, 0, None, None, None) == N.ERR_INVALID_ARG
    st = N.mecuco_stats()
    assert lib.mecuco_get_stats(None, C.byref(st), None) == N.ERR_INVALID_ARG


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2606_06329_gb300 import _native
    with pytest.raises(_native.MecucoNotBuilt):
        saved = _native._lib
        _native._lib = None
        try:
            _native.load(str(tmp_path / "missing.so"))
        finally:
            _native._lib = saved
