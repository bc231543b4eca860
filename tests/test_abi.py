"""Host-side checks of the C ABI library (no GPU needed, no kernel launched)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1802_01359_gb300 import build, fif

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fif.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fif.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fif_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(fif.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(6):
        s = fif.status_string(code)
        assert s.startswith("FIF_")
    assert "unknown" in fif.status_string(99)


def _desc(**kw):
    d = dict(window=0, nu=1.6, mask_scale=1, delta=1e-3, max_inner=200, max_imfs=10, precision=0,
             max_n=4096, flags=0, gamma=0.0)
    d.update(kw)
    return fif.PlanDesc(d["window"], d["nu"], d["mask_scale"], d["delta"], d["max_inner"],
                        d["max_imfs"], d["precision"], d["max_n"], d["flags"], d["gamma"])


@pytest.mark.parametrize("bad", [dict(delta=0.0), dict(delta=-1.0), dict(max_inner=0),
                                 dict(max_imfs=-1), dict(max_imfs=65), dict(max_n=3),
                                 dict(max_n=(1 << 24) + 1), dict(window=7), dict(mask_scale=0),
                                 dict(mask_scale=3), dict(nu=0.0), dict(flags=16), dict(flags=32),
                                 dict(delta=float("nan")), dict(gamma=1.0), dict(gamma=-0.1),
                                 dict(gamma=float("nan"))])
def test_plan_descriptor_validation(lib, bad):
    """Invalid descriptors are rejected before any CUDA call."""
    h = ctypes.c_void_p()
    rc = lib.fif_plan_create(ctypes.byref(h), ctypes.byref(_desc(**bad)), None)
    assert rc == fif.FIF_EINVAL and not h.value


def test_null_arguments(lib):
    assert lib.fif_plan_create(None, ctypes.byref(_desc()), None) == fif.FIF_EINVAL
    h = ctypes.c_void_p()
    assert lib.fif_plan_create(ctypes.byref(h), None, None) == fif.FIF_EINVAL
    assert lib.fif_plan_destroy(None) == fif.FIF_OK
    assert lib.fif_plan_set_stream(None, None) == fif.FIF_EINVAL
    assert lib.fif_plan_prepare(None, None, 0) == fif.FIF_EINVAL
    assert lib.fif_decompose(None, None, 0, None, None, None, None, None, None) == fif.FIF_EINVAL
    assert lib.fif_decompose_batch(None, None, None, 1, None, None, None, None, None, None,
                                   None) == fif.FIF_EINVAL
    assert lib.fif_decompose_batch_host(None, None, None, 1, None, None, None, None, None, None,
                                        None) == fif.FIF_EINVAL


def _shape_desc(g, **kw):
    d = _desc(window=fif.WIN_SHAPE, **kw)
    arr = None
    if g is not None:
        arr = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        d.window_shape = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.window_shape_len = arr.size
    return d, arr


@pytest.mark.parametrize("g", [None, [], [-1.0, 1.0], [1.0, float("nan")], [1.0, 0.0, 1.0], [0.0],
                               [0.0, 0.0], [float("inf")]])
def test_shape_window_validation(lib, g):
    """FIF_WIN_SHAPE needs finite samples >= 0 with an interpolant > 0 inside (0, 1)."""
    d, keep = _shape_desc(g)
    h = ctypes.c_void_p()
    assert lib.fif_plan_create(ctypes.byref(h), ctypes.byref(d), None) == fif.FIF_EINVAL
    assert not h.value


@pytest.mark.parametrize("flags", [fif.APRIORI_N0])
def test_shape_window_unsupported_combinations(lib, flags):
    d, keep = _shape_desc([0.0, 1.0, 0.0], flags=flags)
    h = ctypes.c_void_p()
    assert lib.fif_plan_create(ctypes.byref(h), ctypes.byref(d), None) == fif.FIF_EUNSUPPORTED


def test_shape_window_not_on_the_noalloc_path(lib):
    """The allocation-free entry point has no per-(n, L) table: refused before any CUDA call."""
    d, keep = _shape_desc([1.0])
    dummy = ctypes.c_void_p(16)
    rc = lib.fif_decompose_noalloc(ctypes.byref(d), dummy, 64, dummy, dummy, dummy, dummy, dummy,
                                   None, None)
    assert rc == fif.FIF_EUNSUPPORTED


def test_unknown_precision_rejected(lib):
    """FIF_PREC_FP32 (0) and FIF_PREC_SPLIT_BF16 (1) are the precisions; another value is
    refused before any CUDA call."""
    h = ctypes.c_void_p()
    assert lib.fif_plan_create(ctypes.byref(h), ctypes.byref(_desc(precision=2)), None) == \
        fif.FIF_EINVAL


def test_binding_fails_loudly_without_library(tmp_path):
    saved = fif._lib
    fif._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            fif.load_library(str(tmp_path / "missing.so"))
    finally:
        fif._lib = saved


def test_out_layout():
    import numpy as np
    assert fif.out_layout([4, 6, 8], 2).tolist() == [0, 12, 30]
    assert np.array_equal(fif.out_layout([], 3), np.zeros(0, dtype=np.int64))


def test_batch_launches_rejects_null_arguments(lib):
    v = ctypes.c_int64()
    assert lib.fif_plan_batch_launches(None, ctypes.byref(v)) == fif.FIF_EINVAL


def test_tuning_entry_points_reject_null_arguments(lib):
    i32 = ctypes.c_int32()
    assert lib.fif_plan_tune(None, None, None, 1, None, None, None, None, None, None) == \
        fif.FIF_EINVAL
    assert lib.fif_plan_get_schedule(None, 4096, ctypes.byref(i32), ctypes.byref(i32),
                                     ctypes.byref(i32)) == fif.FIF_EINVAL
    assert lib.fif_plan_save_tuning(None, b"/nonexistent/x") == fif.FIF_EINVAL
    assert lib.fif_plan_load_tuning(None, b"/nonexistent/x") == fif.FIF_EINVAL
