"""The allocation-free forward entry point (fwh_forward_noalloc) against fwh_forward.

Callers that cannot allocate device memory while they run (a real-time loop
with a fixed memory budget, a host callback, code inside a framework that owns
the device memory) use fwh_forward_noalloc, whose scratch is a static device
array.  This file is collected last on purpose.  It calls both entry points
through the C ABI on the same device buffers, twice in a row (the second call
sees the scratch the first one left behind), and checks that an oversized
problem is refused with a clear error instead of running.
"""
import ctypes

import numpy as np
import pytest
import torch

from fwh_inputs import FlowCase, observers_circle, uv_sphere
from fwh_inputs.analytic import surface_fields

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-4}   # rel-L2 per observer, as in the parity tests
DEG = np.pi / 180


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    from paper_2312_16263_gb300 import _abi
    return _abi.load()


def _handle(lib, surf, mach, aoa, dt, prec, obs):
    from paper_2312_16263_gb300 import _abi
    h = ctypes.c_void_p()
    y = np.ascontiguousarray(surf.centroids)
    n = np.ascontiguousarray(surf.normals)
    a = np.ascontiguousarray(surf.areas)
    st = lib.fwh_create(ctypes.byref(h), surf.n_panels, y.ctypes.data, n.ctypes.data,
                        a.ctypes.data, mach, aoa, 1.0 / mach, dt,
                        _abi.FWH_FP64 if prec == "fp64" else _abi.FWH_MIXED)
    _abi.check(st, None)
    x = np.ascontiguousarray(obs)
    _abi.check(lib.fwh_set_observers(h, x.shape[0], x.ctypes.data), h)
    return h


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_matches_forward_twice(lib, prec):
    from paper_2312_16263_gb300 import _abi
    rng = np.random.default_rng(42)
    surf = uv_sphere(1.0, 17, 29)                      # 493 panels (ragged)
    mach, aoa, dt, nt = 0.4, 7 * DEG, 0.03, 389        # ragged record
    obs = observers_circle(30.0, 11) + rng.normal(size=(11, 3))
    f = surface_fields("dipole", surf.centroids, FlowCase(mach, aoa), 0.01, 2 * np.pi, dt, nt)
    f += rng.normal(size=f.shape) * 1e-4
    dt_t = torch.float64 if prec == "fp64" else torch.float32
    fields = torch.as_tensor(f, dtype=dt_t).cuda().contiguous()
    h = _handle(lib, surf, mach, aoa, dt, prec, obs)
    try:
        ref = torch.empty((obs.shape[0], nt), dtype=torch.float64, device="cuda")
        _abi.check(lib.fwh_forward(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                   ctypes.c_void_p(ref.data_ptr()), _stream()), h)
        for call in range(2):
            out = torch.full_like(ref, float("nan"))
            _abi.check(lib.fwh_forward_noalloc(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                               ctypes.c_void_p(out.data_ptr()), _stream()), h)
            torch.cuda.synchronize()
            _abi.check(lib.fwh_check(h, _stream()), h)
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            for o in range(b.shape[0]):
                den = np.linalg.norm(b[o])
                err = np.linalg.norm(a[o] - b[o]) / den if den > 0 else np.abs(a[o]).max()
                assert err <= TOL[prec], (prec, call, o, err)
    finally:
        lib.fwh_destroy(h)


def test_noalloc_rejects_oversized_problem(lib):
    from paper_2312_16263_gb300 import _abi
    surf = uv_sphere(1.0, 64, 128)                     # 8192 panels
    nt = 4096                                          # 8192 x 4096 x 64 B = 2 GiB > 64 MiB
    obs = observers_circle(30.0, 2)
    h = _handle(lib, surf, 0.3, 0.0, 0.02, "mixed", obs)
    try:
        fields = torch.zeros((nt, 5, surf.n_panels), dtype=torch.float32, device="cuda")
        out = torch.zeros((2, nt), dtype=torch.float64, device="cuda")
        st = lib.fwh_forward_noalloc(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                     ctypes.c_void_p(out.data_ptr()), _stream())
        assert st == _abi.FWH_ERR_ARG
        assert b"static scratch holds" in lib.fwh_last_error(h)
        # host buffers are refused too (the call never stages)
        hf = torch.zeros((16, 5, surf.n_panels), dtype=torch.float32)
        ho = torch.zeros((2, 16), dtype=torch.float64)
        st = lib.fwh_forward_noalloc(h, ctypes.c_void_p(hf.data_ptr()), 16,
                                     ctypes.c_void_p(ho.data_ptr()), _stream())
        assert st == _abi.FWH_ERR_ARG
    finally:
        lib.fwh_destroy(h)
