"""Torch-facing wrapper of the C ABI (device memory and streams from PyTorch).

`FWH` owns one library handle (one permeable surface + flow + observers).
Tensors are passed to the library as raw pointers on the current CUDA stream;
host tensors go through the library's own staging.  Nothing here computes any
part of the FW-H path.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _abi

_PREC = {"fp64": _abi.FWH_FP64, "mixed": _abi.FWH_MIXED}


def _stream_ptr(stream=None):
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _f64_host(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


class FWH:
    """One surface: `FWH(centroids, normals, areas, mach, aoa, dt, precision)`.

    precision: 'fp64' (double fields and arithmetic) or 'mixed' (float fields
    and integrand arithmetic, FP64 arrival times and weights, FP64 output).
    """

    def __init__(self, centroids, normals, areas, mach: float, aoa: float, dt: float,
                 precision: str = "mixed", observers=None):
        self.lib = _abi.load()
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        y, n, dS = _f64_host(centroids), _f64_host(normals), _f64_host(areas)
        self.P = int(dS.shape[0])
        self.mach, self.aoa, self.dt = float(mach), float(aoa), float(dt)
        h = ctypes.c_void_p()
        st = self.lib.fwh_create(ctypes.byref(h), self.P, y.ctypes.data, n.ctypes.data,
                                 dS.ctypes.data, self.mach, self.aoa, 1.0 / self.mach,
                                 self.dt, _PREC[precision])
        _abi.check(st, None)
        self.h = h
        self.O = 0
        if observers is not None:
            self.set_observers(observers)

    @classmethod
    def from_workload(cls, w, precision="mixed"):
        s = w.surface
        return cls(s.centroids, s.normals, s.areas, w.mach, w.aoa, w.dt, precision,
                   observers=w.observers)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fwh_destroy(self.h)
            self.h = None

    __del__ = close

    def set_observers(self, xyz):
        x = _f64_host(xyz).reshape(-1, 3)
        _abi.check(self.lib.fwh_set_observers(self.h, x.shape[0], x.ctypes.data), self.h)
        self.O = int(x.shape[0])

    def window(self, nt: int):
        ts = np.empty(self.O, dtype=np.float64)
        nv = np.empty(self.O, dtype=np.int64)
        _abi.check(self.lib.fwh_observer_window(
            self.h, int(nt), ts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), self.h)
        return ts, nv

    def observer_extremes(self):
        """(R_max, R_min) per observer over this surface's own panels."""
        mx = np.empty(self.O, dtype=np.float64)
        mn = np.empty(self.O, dtype=np.float64)
        _abi.check(self.lib.fwh_observer_extremes(
            self.h, mx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            mn.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.h)
        return mx, mn

    def set_observer_extremes(self, r_max, r_min):
        """Use the given (all-reduced) extremes for the observer window."""
        mx = np.ascontiguousarray(r_max, dtype=np.float64)
        mn = np.ascontiguousarray(r_min, dtype=np.float64)
        _abi.check(self.lib.fwh_set_observer_extremes(
            self.h, mx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            mn.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.h)

    def _check_fields(self, fields: torch.Tensor):
        if fields.dtype != self.dtype:
            raise TypeError(f"fields must be {self.dtype} for precision {self.precision}")
        if fields.dim() != 3 or fields.shape[1] != 5 or fields.shape[2] != self.P:
            raise ValueError(f"fields must be [nt][5][{self.P}], got {tuple(fields.shape)}")
        if not fields.is_contiguous():
            raise ValueError("fields must be contiguous")

    def forward(self, fields: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """p_out [O][nt] float64 on the fields' device (host fields -> host output).

        A device-side check that fails during a call with device outputs is
        raised (FWHError) by the next call on this surface, or by check()."""
        self._check_fields(fields)
        nt = fields.shape[0]
        if out is None:
            out = torch.empty((self.O, nt), dtype=torch.float64, device=fields.device)
        _abi.check(self.lib.fwh_forward(self.h, ctypes.c_void_p(fields.data_ptr()), nt,
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
                   self.h)
        return out

    def backward(self, fields: torch.Tensor, grad_p: torch.Tensor,
                 out: torch.Tensor | None = None, stream=None):
        """dLoss/dfields [nt][5][P] (fields' dtype) from dLoss/dp_out [O][nt]."""
        self._check_fields(fields)
        nt = fields.shape[0]
        grad_p = grad_p.to(dtype=torch.float64).contiguous()
        if out is None:
            out = torch.empty_like(fields)
        _abi.check(self.lib.fwh_backward(self.h, ctypes.c_void_p(fields.data_ptr()), nt,
                                         ctypes.c_void_p(grad_p.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
                   self.h)
        return out

    def autotune(self, nt: int, stream=None) -> int:
        c = ctypes.c_int(-1)
        _abi.check(self.lib.fwh_autotune(self.h, int(nt), ctypes.byref(c), _stream_ptr(stream)),
                   self.h)
        return int(c.value)

    def set_tile_config(self, idx: int):
        _abi.check(self.lib.fwh_set_tile_config(self.h, int(idx)), self.h)

    def set_wait_limit(self, cycles: int = 0, withhold_copies: bool = False):
        """Bound (SM clocks) of the forward pipeline's waits; 0 = default.
        withhold_copies (testing): issue no copies, so every wait runs out."""
        _abi.check(self.lib.fwh_set_wait_limit(self.h, int(cycles), int(bool(withhold_copies))),
                   self.h)

    def set_pipeline(self, enable: bool = True):
        """Overlap the series prep of later time segments with the scatter."""
        _abi.check(self.lib.fwh_set_pipeline(self.h, int(bool(enable))), self.h)

    def set_batch_options(self, ring: int = 0, form: str = "pipelined"):
        """Options of batched calls this surface leads (first in the list):
        ring = 0 keeps whole records, > 0 streams them through a ring of that
        many source samples (whole 512-sample segments, at least one); form
        is "pipelined" (one launch per surface, preps overlapped), "grid" (one
        grid over every surface) or "persistent" (the work-queue kernel)."""
        forms = {"pipelined": _abi.FWH_BATCH_PIPELINED, "grid": _abi.FWH_BATCH_GRID,
                 "persistent": _abi.FWH_BATCH_PERSISTENT}
        _abi.check(self.lib.fwh_set_batch_options(self.h, int(ring), forms[form]), self.h)

    def set_timing(self, enable: bool = True):
        _abi.check(self.lib.fwh_set_timing(self.h, int(bool(enable))), self.h)

    def last_timings(self):
        ms = (ctypes.c_float * 3)()
        _abi.check(self.lib.fwh_last_timings(self.h, ms), self.h)
        return {"prep_ms": ms[0], "forward_ms": ms[1], "total_ms": ms[2]}

    def timing_totals(self, reset: bool = True):
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_int64(0)
        _abi.check(self.lib.fwh_timing_totals(self.h, ms, ctypes.byref(n), int(bool(reset))),
                   self.h)
        return {"prep_ms": ms[0], "forward_ms": ms[1], "total_ms": ms[2], "calls": int(n.value)}

    def check(self, stream=None):
        _abi.check(self.lib.fwh_check(self.h, _stream_ptr(stream)), self.h)


def welch_psd(p: torch.Tensor, fs: float, nperseg: int, n_valid=None, detrend: bool = True,
              span_ratio: float = 1.0, p_ref: float = 0.0, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """Span-corrected Welch PSD of each row of p [n_sig][ld] (fwh_psd; Sec. IV C,
    Eq. PSD_corr).  n_valid: samples per row (e.g. FWH.window(nt)[1]) or None.
    Returns [n_sig][nperseg // 2 + 1] float64 on p's device."""
    if p.dtype != torch.float64 or p.dim() != 2 or not p.is_contiguous():
        raise ValueError("p must be a contiguous [n_sig][ld] float64 tensor")
    n_sig, ld = p.shape
    if out is None:
        out = torch.empty((n_sig, nperseg // 2 + 1), dtype=torch.float64, device=p.device)
    nv = None
    if n_valid is not None:
        nv = torch.as_tensor(np.asarray(n_valid, dtype=np.int64) if not isinstance(
            n_valid, torch.Tensor) else n_valid, dtype=torch.int64).contiguous()
    lib = _abi.load()
    _abi.check(lib.fwh_psd(n_sig, ctypes.c_void_p(p.data_ptr()), ld,
                           ctypes.c_void_p(nv.data_ptr()) if nv is not None else None,
                           float(fs), int(nperseg), int(bool(detrend)), float(span_ratio),
                           float(p_ref), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def moving_forward(y: torch.Tensor, normals: torch.Tensor, velocities: torch.Tensor,
                   areas, c0: float, rho0: float, dt: float, fields: torch.Tensor, x0,
                   w=(0.0, 0.0, 0.0), out: torch.Tensor | None = None, stream=None):
    """General moving surface (fwh_forward_moving; Eqs. pT, pL of Sec. II B).

    y, normals, velocities [nt][P][3], fields [nt][5][P] float64 on one
    device; observers at x0 [O][3] moving with w.  Returns (p_out [O][nt] on
    the fields' device, t_start [O], n_valid [O])."""
    nt, P = fields.shape[0], fields.shape[2]
    for t in (y, normals, velocities):
        if t.dtype != torch.float64 or tuple(t.shape) != (nt, P, 3) or not t.is_contiguous():
            raise ValueError("y, normals, velocities must be contiguous [nt][P][3] float64")
    if fields.dtype != torch.float64 or not fields.is_contiguous():
        raise ValueError("fields must be contiguous [nt][5][P] float64")
    dev = fields.device
    dS = torch.as_tensor(np.asarray(areas, dtype=np.float64), device=dev).contiguous()
    x = torch.as_tensor(np.asarray(x0, dtype=np.float64).reshape(-1, 3), device=dev).contiguous()
    ww = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(3))
    O = x.shape[0]
    if out is None:
        out = torch.empty((O, nt), dtype=torch.float64, device=dev)
    ts = np.empty(O, dtype=np.float64)
    nv = np.empty(O, dtype=np.int64)
    lib = _abi.load()
    _abi.check(lib.fwh_forward_moving(
        P, nt, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(normals.data_ptr()),
        ctypes.c_void_p(velocities.data_ptr()), ctypes.c_void_p(dS.data_ptr()), float(c0),
        float(rho0), float(dt), ctypes.c_void_p(fields.data_ptr()), O,
        ctypes.c_void_p(x.data_ptr()), ww.ctypes.data, ctypes.c_void_p(out.data_ptr()),
        ts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _stream_ptr(stream)))
    return out, ts, nv


def batch_forward(surfaces: Sequence[FWH], fields: Sequence[torch.Tensor],
                  outs: Sequence[torch.Tensor] | None = None, stream=None):
    """Several surfaces in one graph-captured call (launch form and series
    ring set on surfaces[0] with set_batch_options)."""
    n = len(surfaces)
    if outs is None:
        outs = [torch.empty((s.O, f.shape[0]), dtype=torch.float64, device=f.device)
                for s, f in zip(surfaces, fields)]
    for s, f in zip(surfaces, fields):
        s._check_fields(f)
    hs = (ctypes.c_void_p * n)(*[s.h.value for s in surfaces])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fields])
    op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    nts = (ctypes.c_int64 * n)(*[f.shape[0] for f in fields])
    lib = _abi.load()
    _abi.check(lib.fwh_batch_forward(n, hs, fp, nts, op, _stream_ptr(stream)), surfaces[0].h)
    return outs
