"""The C ABI library builds, loads without a GPU and exports every entry point of include/pdd.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pdd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdd_[A-Za-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_08946_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("pdd_build_cover", "pdd_assemble_G", "pdd_solve", "pdd_grad", "pdd_system_csr",
                 "pdd_destroy_cover", "pdd_destroy_system", "pdd_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_export():
    import paper_2311_08946_gb300 as pkg
    assert set(_declared()) <= set(pkg.EXPORTS) | {"pdd_version"}


def test_version_and_launch_counter_without_gpu(lib):
    lib.pdd_version.restype = ctypes.c_char_p
    lib.pdd_launch_count.restype = ctypes.c_int64
    assert b"sm_103a" in lib.pdd_version()
    assert lib.pdd_launch_count() >= 0


def test_invalid_arguments_rejected_before_any_device_work(lib):
    import paper_2311_08946_gb300 as pkg
    pkg.load()
    h = ctypes.c_void_p()
    # null domain -> PDD_EINVAL, with a message
    st = pkg._lib.pdd_build_cover(None, None, ctypes.byref(h), None)
    assert st == 1
    assert b"domain" in pkg._lib.pdd_last_error()
    dom = pkg._Domain(0, (ctypes.c_double * 4)(0, 0, 1, 1))
    spec = pkg._CoverSpec(0, 4, 4, 0.125, 0.125, 0.25, 0.2, 15, 16, 16, 0, None, None, None, None, None, None)
    st = pkg._lib.pdd_build_cover(ctypes.byref(dom), ctypes.byref(spec), ctypes.byref(h), None)
    assert st == 1 and b"n_knots" in pkg._lib.pdd_last_error()
    bad_dom = pkg._Domain(0, (ctypes.c_double * 4)(1, 0, 0, 1))
    st = pkg._lib.pdd_build_cover(ctypes.byref(bad_dom), ctypes.byref(spec), ctypes.byref(h), None)
    assert st == 1
    so = pkg._SolveOpts(0, 10, 1e-10, 0)
    st = pkg._lib.pdd_solve_csr(4, None, None, None, None, None, ctypes.byref(so), None, None)
    assert st == 1


def test_new_entry_points_reject_bad_arguments_without_gpu(lib):
    """The row mode, the Eq. 46 families and the new accessors are validated on the host."""
    import paper_2311_08946_gb300 as pkg
    pkg.load()
    h = ctypes.c_void_p()
    dom = pkg._Domain(0, (ctypes.c_double * 4)(0, 0, 1, 1))
    spec = pkg._CoverSpec(0, 4, 4, 0.125, 0.125, 0.25, 0.2, 16, 16, 16, 0, None, None, None, None, None, None, 7)
    st = pkg._lib.pdd_build_cover(ctypes.byref(dom), ctypes.byref(spec), ctypes.byref(h), None)
    assert st == 1 and b"row mode" in pkg._lib.pdd_last_error()
    n = ctypes.c_int()
    pp = ctypes.c_void_p()
    assert pkg._lib.pdd_cover_rows(None, ctypes.byref(n), ctypes.byref(pp), ctypes.byref(pp)) == 1
    assert pkg._lib.pdd_system_mc_subs(None, ctypes.byref(pp)) == 1
    assert pkg.ROW_MODE == {"farthest": 0, "averaged": 1}
    assert pkg._F["eq46"] == 3 and pkg._G["eq46"] == 5

