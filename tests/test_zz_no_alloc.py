"""The allocation-free forward entry point (fwh_forward_noalloc) against fwh_forward.

Callers that cannot allocate device memory while they run (a real-time loop
with a fixed memory budget, code inside a framework that owns the device
memory) use fwh_forward_noalloc, whose scratch is a static device array.  This
file is collected last on purpose.  It calls both entry points through the C
ABI on the same device buffers, twice in a row (the second call sees the
scratch the first one left behind, and must not change the device's
allocations), checks that the handle still plans, runs forward and backward
correctly under another tile shape afterwards, and that an oversized problem
is refused with a clear error instead of running.
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
        outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        for call in range(2):
            out = outs[call]
            if call == 1:
                alloc0 = torch.cuda.memory_allocated()
                free0, _ = torch.cuda.mem_get_info()
            _abi.check(lib.fwh_forward_noalloc(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                               ctypes.c_void_p(out.data_ptr()), _stream()), h)
            torch.cuda.synchronize()
            if call == 1:  # the steady-state call allocated nothing on the device
                assert torch.cuda.memory_allocated() == alloc0
                assert torch.cuda.mem_get_info()[0] == free0
            _abi.check(lib.fwh_check(h, _stream()), h)
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            for o in range(b.shape[0]):
                den = np.linalg.norm(b[o])
                err = np.linalg.norm(a[o] - b[o]) / den if den > 0 else np.abs(a[o]).max()
                assert err <= TOL[prec], (prec, call, o, err)
    finally:
        lib.fwh_destroy(h)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_handle_after_noalloc_other_shape(lib, prec):
    """After fwh_forward_noalloc, a switch to another tile shape re-plans the
    handle, and fwh_forward / fwh_backward still agree with the oracle."""
    from oracle import Oracle
    from paper_2312_16263_gb300 import _abi
    rng = np.random.default_rng(7)
    surf = uv_sphere(1.0, 13, 27)                      # 351 panels
    mach, aoa, dt, nt = 0.45, -4 * DEG, 0.03, 301
    obs = observers_circle(25.0, 5) + rng.normal(size=(5, 3))
    f = surface_fields("monopole", surf.centroids, FlowCase(mach, aoa), 0.01, 2 * np.pi, dt, nt)
    f += rng.normal(size=f.shape) * 1e-4
    dt_t = torch.float64 if prec == "fp64" else torch.float32
    fields = torch.as_tensor(f, dtype=dt_t).cuda().contiguous()
    h = _handle(lib, surf, mach, aoa, dt, prec, obs)
    try:
        out = torch.empty((obs.shape[0], nt), dtype=torch.float64, device="cuda")
        _abi.check(lib.fwh_forward_noalloc(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                           ctypes.c_void_p(out.data_ptr()), _stream()), h)
        _abi.check(lib.fwh_set_tile_config(h, 1), h)   # another shape: another plan
        p = torch.empty_like(out)
        _abi.check(lib.fwh_forward(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                   ctypes.c_void_p(p.data_ptr()), _stream()), h)
        orc = Oracle(surf.centroids, surf.normals, surf.areas, mach, aoa, dt)
        fd = fields.double().cpu().numpy()
        p_ref, _, nv_ref = orc.forward(fd, obs)
        ts = np.empty(obs.shape[0])
        nv = np.empty(obs.shape[0], dtype=np.int64)
        _abi.check(lib.fwh_observer_window(
            h, nt, ts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), h)
        gm = rng.normal(size=(obs.shape[0], nt))
        for o in range(obs.shape[0]):  # both sides ignore entries past their own N_o
            gm[o, min(nv[o], nv_ref[o]):] = 0.0
        g_p = torch.as_tensor(gm, dtype=torch.float64, device="cuda")
        g = torch.empty_like(fields)
        _abi.check(lib.fwh_backward(h, ctypes.c_void_p(fields.data_ptr()), nt,
                                    ctypes.c_void_p(g_p.data_ptr()),
                                    ctypes.c_void_p(g.data_ptr()), _stream()), h)
        torch.cuda.synchronize()
        _abi.check(lib.fwh_check(h, _stream()), h)
        a, b = p.cpu().numpy(), out.cpu().numpy()
        for o in range(obs.shape[0]):
            n = int(min(nv[o], nv_ref[o]))
            den = np.linalg.norm(p_ref[o, :n])
            assert np.linalg.norm(a[o, :n] - p_ref[o, :n]) / den <= TOL[prec], (prec, o)
            assert np.linalg.norm(b[o, :n] - p_ref[o, :n]) / den <= TOL[prec], (prec, o)
        g_ref = orc.backward(fd, obs, gm)
        gg = g.double().cpu().numpy()
        assert np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref) <= \
            (1e-9 if prec == "fp64" else 1e-4)
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
