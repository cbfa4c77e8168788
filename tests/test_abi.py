"""The C-ABI library builds, loads and exports every symbol include/fwh.h declares
(CPU only: no compute call is made), and argument validation needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_16263_gb300.build import build
    build()
    from paper_2312_16263_gb300 import _abi
    return _abi.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fwh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwh_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("fwh_create", "fwh_set_observers", "fwh_forward", "fwh_backward",
              "fwh_batch_forward", "fwh_observer_window", "fwh_destroy", "fwh_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2312_16263_gb300 import _abi
    for s in declared_symbols():
        assert hasattr(lib, s), s
        assert s in _abi.SIGNATURES, f"binding lacks {s}"


def test_binding_names_match_header():
    from paper_2312_16263_gb300 import _abi
    assert sorted(_abi.SIGNATURES) == declared_symbols()


def test_argument_validation_without_gpu(lib):
    from paper_2312_16263_gb300 import _abi
    h = ctypes.c_void_p()
    y = np.zeros((4, 3))
    n = np.tile([1.0, 0.0, 0.0], (4, 1))
    a = np.ones(4)
    P = ctypes.c_void_p
    # mach outside (0, 1)
    st = lib.fwh_create(ctypes.byref(h), 4, y.ctypes.data, n.ctypes.data, a.ctypes.data,
                        1.2, 0.0, 1 / 1.2, 0.1, 0)
    assert st == _abi.FWH_ERR_ARG and b"mach" in lib.fwh_last_error(None)
    # c0 inconsistent with mach
    st = lib.fwh_create(ctypes.byref(h), 4, y.ctypes.data, n.ctypes.data, a.ctypes.data,
                        0.3, 0.0, 340.0, 0.1, 0)
    assert st == _abi.FWH_ERR_ARG and b"c0" in lib.fwh_last_error(None)
    # non-unit normal
    bad = n.copy()
    bad[2] = [2.0, 0, 0]
    st = lib.fwh_create(ctypes.byref(h), 4, y.ctypes.data, bad.ctypes.data, a.ctypes.data,
                        0.3, 0.0, 1 / 0.3, 0.1, 0)
    assert st == _abi.FWH_ERR_ARG and b"normal" in lib.fwh_last_error(None)
    # zero area, bad precision, dt <= 0, null pointers
    z = a.copy()
    z[1] = 0
    assert lib.fwh_create(ctypes.byref(h), 4, y.ctypes.data, n.ctypes.data, z.ctypes.data,
                          0.3, 0.0, 1 / 0.3, 0.1, 0) == _abi.FWH_ERR_ARG
    assert lib.fwh_create(ctypes.byref(h), 4, y.ctypes.data, n.ctypes.data, a.ctypes.data,
                          0.3, 0.0, 1 / 0.3, 0.1, 7) == _abi.FWH_ERR_ARG
    assert lib.fwh_create(ctypes.byref(h), 4, y.ctypes.data, n.ctypes.data, a.ctypes.data,
                          0.3, 0.0, 1 / 0.3, -0.1, 0) == _abi.FWH_ERR_ARG
    assert lib.fwh_create(ctypes.byref(h), 4, None, n.ctypes.data, a.ctypes.data,
                          0.3, 0.0, 1 / 0.3, 0.1, 0) == _abi.FWH_ERR_ARG
    assert lib.fwh_create(None, 4, y.ctypes.data, n.ctypes.data, a.ctypes.data,
                          0.3, 0.0, 1 / 0.3, 0.1, 0) == _abi.FWH_ERR_ARG
    # NULL handle everywhere
    assert lib.fwh_set_observers(None, 1, y.ctypes.data) == _abi.FWH_ERR_ARG
    assert lib.fwh_forward(None, P(1), 10, P(1), None) == _abi.FWH_ERR_ARG
    assert lib.fwh_backward(None, P(1), 10, P(1), P(1), None) == _abi.FWH_ERR_ARG
    assert lib.fwh_batch_forward(0, None, None, None, None, None) == _abi.FWH_ERR_ARG
    assert lib.fwh_set_batch_options(None, 0, _abi.FWH_BATCH_GRID) == _abi.FWH_ERR_ARG
    assert lib.fwh_set_moving_scratch(-1) == _abi.FWH_ERR_ARG
    lib.fwh_destroy(None)
    assert lib.fwh_version().startswith(b"fwh-gb300")


def test_package_fails_loudly_without_library(tmp_path):
    import paper_2312_16263_gb300._abi as m
    saved = m._lib
    try:
        m._lib = None
        with pytest.raises(ImportError):
            m.load(str(tmp_path / "missing.so"))
    finally:
        m._lib = saved
