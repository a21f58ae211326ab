"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports every
function include/mca.h declares; the ctypes records match the header's layout."""
import ctypes
import os
import re

import pytest

import paper_2109_07929_gb300 as mca

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "mca.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mca_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = _declared()
    assert set(mca.EXPORTED) <= set(names)
    assert "mca_solve" in names and "mca_create" in names


def test_library_exports_every_declared_symbol():
    lib = mca.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts():
    # mca_params: 2 int32, 7 doubles, 4 int32, 3 doubles, 2 int32
    assert ctypes.sizeof(mca.Params) == 8 + 7 * 8 + 4 * 4 + 3 * 8 + 8 + 8
    assert ctypes.sizeof(mca.Stats) == 4 * 4 + 2 * 8


def test_default_params_and_errors_without_gpu():
    lib = mca.load()
    p = mca.default_params(4, 5)
    assert p.precision == mca.PREC_BF16_SPLIT and p.gmres_restart == 30
    assert p.g_src == 0.1 and p.g_term_top_right == 1e-3 and p.b == 2.0
    assert lib.mca_strerror(mca.ERR_TIMEOUT).decode().startswith("bounded")
    # invalid sizes are rejected before any device work
    p.rows = 0
    h = ctypes.c_void_p()
    import numpy as np
    g = np.ones(20)
    rc = lib.mca_create(ctypes.byref(p), g.ctypes.data, ctypes.byref(h))
    assert rc == mca.ERR_INVALID_ARG
    assert lib.mca_solve(None, None, 0, None, None, None, None, None) == mca.ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [
    ("rows", 16385), ("cols", 0), ("g_wire_top", 0.0), ("g_sense", float("inf")),
    ("b", -1.0), ("b", float("nan")), ("device_model", 9), ("precision", 99),
    ("gmres_restart", 0), ("gmres_restart", 31), ("max_batch", 0), ("max_batch", 65),
    ("max_newton", 0), ("flags", 0x100), ("newton_rtol", 0.0), ("eta0", -1.0)])
def test_create_rejects_each_invalid_parameter_before_device_work(field, value):
    """mca_create validates every parameter on the host and returns MCA_ERR_INVALID_ARG
    with a message, before touching the device (so this runs without a GPU)."""
    import numpy as np
    lib = mca.load()
    p = mca.default_params(4, 5)
    setattr(p, field, value)
    h = ctypes.c_void_p()
    g = np.ones(20)
    assert lib.mca_create(ctypes.byref(p), g.ctypes.data, ctypes.byref(h)) == mca.ERR_INVALID_ARG
    assert not h.value
    assert lib.mca_last_error_message().decode() != ""


def test_yakopcic_needs_a_positive_ratio():
    import numpy as np
    lib = mca.load()
    p = mca.default_params(3, 3, device_model=mca.DEVICE_YAKOPCIC, neg_ratio=0.0)
    h = ctypes.c_void_p()
    g = np.ones(9)
    assert lib.mca_create(ctypes.byref(p), g.ctypes.data, ctypes.byref(h)) == mca.ERR_INVALID_ARG
