"""The C ABI library loads on a machine without a GPU and exports every entry
point that include/spc5.h declares. Only host-side argument checks are
exercised here (they return before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_1801_01134_gb300 import _build, spc5

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(spc5_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return spc5.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spc5_convert", "spc5_spmv", "spc5_spmv_acc", "spc5_export", "spc5_destroy", "spc5_last_error",
                 "spc5_count_blocks", "spc5_csr_spmv", "spc5_copy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_host_side_argument_checks(lib):
    h = ctypes.c_void_p()
    # NULL output handle
    assert lib.spc5_convert(4, 4, 0, None, None, None, 0, 1, 8, None, None, None) == spc5.EINVAL
    # unsupported block shape / value type, negative sizes, index range
    assert lib.spc5_convert(4, 4, 0, 1, None, None, 0, 3, 8, None, None, ctypes.byref(h)) == spc5.EUNSUPPORTED
    assert lib.spc5_convert(4, 4, 0, 1, None, None, 0, 2, 5, None, None, ctypes.byref(h)) == spc5.EUNSUPPORTED
    assert lib.spc5_convert(4, 4, 0, 1, None, None, 7, 2, 8, None, None, ctypes.byref(h)) == spc5.EUNSUPPORTED
    assert lib.spc5_convert(-1, 4, 0, 1, None, None, 0, 2, 8, None, None, ctypes.byref(h)) == spc5.EINVAL
    assert lib.spc5_convert(4, 2**31, 0, 1, None, None, 0, 2, 8, None, None, ctypes.byref(h)) == spc5.ERANGE
    assert lib.spc5_convert(4, 4, 3, 1, None, None, 0, 2, 8, None, None, ctypes.byref(h)) == spc5.EINVAL
    assert "NULL" in spc5.last_error()
    assert lib.spc5_spmv(None, None, None, None) == spc5.EINVAL
    assert lib.spc5_export(None, None) == spc5.EINVAL
    assert lib.spc5_destroy(None) == spc5.OK
    assert lib.spc5_copy(None, None, 17, None) == spc5.EINVAL
    assert lib.spc5_copy(8, 16, 16, None) == spc5.EINVAL  # misaligned
    assert lib.spc5_csr_spmv(4, 4, 0, 1, None, None, 0, 1, 1, 3, None) == spc5.EINVAL  # bad group
    out = (ctypes.c_int64 * 12)()
    assert lib.spc5_count_blocks(4, 4, 0, None, None, out, None) == spc5.EINVAL
    # kernel variants: unknown numbers, and the two-lane form on r > 1, refused before any device work
    for v, r, code in ((2, 1, spc5.EINVAL), (11, 1, spc5.EINVAL), (20, 1, spc5.EINVAL), (34, 1, spc5.EINVAL),
                       (22, 2, spc5.EUNSUPPORTED), (22, 8, spc5.EUNSUPPORTED), (23, 4, spc5.EUNSUPPORTED),
                       (30, 2, spc5.EUNSUPPORTED), (31, 8, spc5.EUNSUPPORTED),
                       (32, 2, spc5.EUNSUPPORTED), (32, 4, spc5.EUNSUPPORTED), (33, 8, spc5.EUNSUPPORTED)):
        opts = spc5.Opts(0, 0, v, 0)
        assert lib.spc5_convert(4, 4, 0, 1, None, None, 0, r, 8, ctypes.byref(opts), None, ctypes.byref(h)) == code, v
    assert lib.spc5_set_variant(None, 22, None) == spc5.EINVAL
    # the tuner checks its arguments before any device work
    res = spc5.TuneResult()
    assert lib.spc5_tune(4, 4, 0, 1, None, None, 0, 0, 3, 0, None, None) == spc5.EINVAL  # no output
    assert lib.spc5_tune(4, 4, 0, 1, None, None, 0, 0, 0, 0, ctypes.byref(res), None) == spc5.EINVAL  # reps
    assert lib.spc5_tune(4, 4, 0, 1, None, None, 0, 2000, 3, 0, ctypes.byref(res), None) == spc5.EINVAL  # k
    assert lib.spc5_tune(4, 4, 0, 1, None, None, 0, 0, 3, 4, ctypes.byref(res), None) == spc5.EINVAL  # flag
    assert lib.spc5_tune(4, 4, 0, None, None, None, 0, 0, 3, 0, ctypes.byref(res), None) == spc5.EINVAL
    assert lib.spc5_tune(4, 4, 0, 1, None, None, 9, 0, 3, 0, ctypes.byref(res), None) == spc5.EUNSUPPORTED
    assert lib.spc5_tune_cache_clear() == spc5.OK
    # the CSR plan and the pool
    plan = ctypes.c_void_p()
    assert lib.spc5_csr_plan_create(4, 0, None, 0, 0, 0, 0, None, ctypes.byref(plan)) == spc5.EINVAL  # no rowptr
    assert lib.spc5_csr_plan_create(4, 0, 1, 0, 3, 0, 0, None, ctypes.byref(plan)) == spc5.EINVAL  # group
    assert lib.spc5_csr_plan_create(4, 0, 1, 0, 0, -1, 0, None, ctypes.byref(plan)) == spc5.EINVAL
    assert lib.spc5_csr_plan_create(4, 0, 1, 7, 0, 0, 0, None, ctypes.byref(plan)) == spc5.EUNSUPPORTED
    assert lib.spc5_csr_spmv_plan(None, None, None, None, None, None) == spc5.EINVAL
    assert lib.spc5_csr_plan_destroy(None) == spc5.OK
    st = ctypes.c_void_p()
    assert lib.spc5_sm_stream_create(0, ctypes.byref(st), None) == spc5.EINVAL
    assert lib.spc5_sm_stream_create(8, None, None) == spc5.EINVAL
    assert lib.spc5_sm_stream_destroy(None) == spc5.OK
    assert lib.spc5_mlp_nparams_n(16) == 6028 and lib.spc5_mlp_nparams_n(20) == 6028 + 4 * 64
    assert lib.spc5_mlp_nparams_n(17) == -1
    f20 = (ctypes.c_double * 20)()
    assert lib.spc5_features_ext(4, 4, 0, 1, None, ctypes.c_double(0.0), f20, None) == spc5.EINVAL  # sm_frac
    assert lib.spc5_mlp_infer_n(None, None, 1, 16, None, None) == spc5.EINVAL
    assert lib.spc5_convert_rows(4, 4, 0, 1, None, None, 0, 2, 8, 1, 4, None, None, ctypes.byref(h)) == spc5.EINVAL
    assert lib.spc5_autotune(None, None, None, 3, None, None, None) == spc5.EINVAL


def test_product_path_has_no_cpu_fallback():
    # the binding never imports the oracle
    src = open(os.path.join(ROOT, "paper_1801_01134_gb300", "spc5.py")).read()
    assert "oracle" not in src.replace("no CPU fallback", "")
    for f in os.listdir(os.path.join(ROOT, "paper_1801_01134_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_1801_01134_gb300", "csrc", f)).read()
