"""ctypes wrapper of the FP64 CPU oracle (oracle/fwh_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg use it; the product library never does.

`build_oracle()` compiles the C source with gcc (-O2, OpenMP, no fused
multiply-add contraction so x86 and Arm round alike) into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfwh_oracle.so")
_lock = threading.Lock()
_handle = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int64)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def load_oracle():
    global _handle
    with _lock:
        if _handle is None:
            lib = ctypes.CDLL(build_oracle())
            sigs = {
                "fwho_convected_distance": [ctypes.c_int64, _D, ctypes.c_double,
                                            ctypes.c_double, _D, _D, _D],
                "fwho_fd_derivative": [ctypes.c_int64, ctypes.c_double, _D, _D],
                "fwho_natural_spline_moments": [ctypes.c_int64, ctypes.c_double, _D, _D],
                "fwho_spline_eval": [ctypes.c_int64, ctypes.c_double, _D, _D,
                                     ctypes.c_int64, _D, _D],
                "fwho_integrands": [ctypes.c_int64, ctypes.c_int64, _D, ctypes.c_double,
                                    _D, _D],
                "fwho_integrands_vjp": [ctypes.c_int64, ctypes.c_int64, _D,
                                        ctypes.c_double, _D, _D, _D],
                "fwho_forward": [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int64, _D,
                                 ctypes.c_int64, _D, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int, ctypes.c_int, _D, _D, _I],
                "fwho_forward_QL": [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int64, _D,
                                    ctypes.c_int64, _D, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, _D, _D, _I],
                "fwho_backward_QL": [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                     ctypes.c_int64, _D, _D, ctypes.c_int, _D],
                "fwho_backward": [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int64, _D,
                                  ctypes.c_int64, _D, _D, ctypes.c_int, _D],
                "fwho_observer_window": [ctypes.c_int64, _D, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                         ctypes.c_int64, _D, _D, _I],
                "fwho_forward_moving": [ctypes.c_int64, ctypes.c_int64, _D, _D, _D, _D,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, _D,
                                        ctypes.c_int64, _D, _D, ctypes.c_int, _D, _D, _I],
                "fwho_max_threads": [],
            }
            for name, args in sigs.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _handle = lib
    return _handle


def _d(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


class Oracle:
    """FP64 oracle bound to one surface + flow; every method is plain CPU code."""

    def __init__(self, centroids, normals, areas, mach, aoa, dt):
        self.lib = load_oracle()
        self.y = _c64(centroids).reshape(-1, 3)
        self.n = _c64(normals).reshape(-1, 3)
        self.dS = _c64(areas).reshape(-1)
        self.P = self.dS.shape[0]
        self.mach, self.aoa, self.dt = float(mach), float(aoa), float(dt)

    @classmethod
    def from_workload(cls, w):
        s = w.surface
        return cls(s.centroids, s.normals, s.areas, w.mach, w.aoa, w.dt)

    # -- building blocks (exposed for pin tests) --------------------------
    def convected_distance(self, d):
        d = _c64(d).reshape(-1, 3)
        n = d.shape[0]
        R, Rs, Rh = np.empty(n), np.empty(n), np.empty((n, 3))
        _check(self.lib.fwho_convected_distance(n, _d(d), self.mach, self.aoa, _d(R),
                                                _d(Rs), _d(Rh)), "convected_distance")
        return R, Rs, Rh

    def integrands(self, fields):
        f = _c64(fields)
        nt = f.shape[0]
        QL = np.empty((nt, 4, self.P))
        _check(self.lib.fwho_integrands(self.P, nt, _d(self.n), self.aoa, _d(f), _d(QL)),
               "integrands")
        return QL

    def integrands_vjp(self, fields, QL_bar):
        f, qb = _c64(fields), _c64(QL_bar)
        out = np.zeros_like(f)
        _check(self.lib.fwho_integrands_vjp(self.P, f.shape[0], _d(self.n), self.aoa,
                                            _d(f), _d(qb), _d(out)), "integrands_vjp")
        return out

    def window(self, obs, nt):
        x = _c64(obs).reshape(-1, 3)
        O = x.shape[0]
        ts, nv = np.empty(O), np.empty(O, dtype=np.int64)
        _check(self.lib.fwho_observer_window(self.P, _d(self.y), self.mach, self.aoa,
                                             self.dt, nt, O, _d(x), _d(ts),
                                             nv.ctypes.data_as(_I)), "window")
        return ts, nv

    # -- the path ------------------------------------------------------------
    def forward(self, fields, obs, p_range=None, compensated=False, threads=0):
        """p_out [O][nt] (zeros at j >= N_o), t_start [O], n_valid [O]."""
        f = _c64(fields)
        nt = f.shape[0]
        assert f.shape == (nt, 5, self.P), f.shape
        return self._fwd(self.lib.fwho_forward, f, nt, obs, p_range, compensated, threads)

    def forward_QL(self, QL, obs, p_range=None, compensated=False, threads=0):
        q = _c64(QL)
        nt = q.shape[0]
        assert q.shape == (nt, 4, self.P), q.shape
        return self._fwd(self.lib.fwho_forward_QL, q, nt, obs, p_range, compensated, threads)

    def _fwd(self, fn, arr, nt, obs, p_range, compensated, threads):
        x = _c64(obs).reshape(-1, 3)
        O = x.shape[0]
        lo, hi = (0, self.P) if p_range is None else p_range
        p_out = np.empty((O, nt))
        ts, nv = np.empty(O), np.empty(O, dtype=np.int64)
        _check(fn(self.P, _d(self.y), _d(self.n), _d(self.dS), self.mach, self.aoa,
                  self.dt, nt, _d(arr), O, _d(x), int(lo), int(hi), int(bool(compensated)),
                  int(threads), _d(p_out), _d(ts), nv.ctypes.data_as(_I)), "forward")
        return p_out, ts, nv

    def backward_QL(self, grad_p, obs, nt, threads=0):
        x = _c64(obs).reshape(-1, 3)
        g = _c64(grad_p)
        out = np.empty((nt, 4, self.P))
        _check(self.lib.fwho_backward_QL(self.P, _d(self.y), _d(self.n), _d(self.dS),
                                         self.mach, self.aoa, self.dt, nt, x.shape[0],
                                         _d(x), _d(g), int(threads), _d(out)), "backward_QL")
        return out

    def backward(self, fields, obs, grad_p, threads=0):
        f = _c64(fields)
        x = _c64(obs).reshape(-1, 3)
        g = _c64(grad_p)
        out = np.empty_like(f)
        _check(self.lib.fwho_backward(self.P, _d(self.y), _d(self.n), _d(self.dS),
                                      self.mach, self.aoa, self.dt, f.shape[0], _d(f),
                                      x.shape[0], _d(x), _d(g), int(threads), _d(out)),
               "backward")
        return out

    # -- textbook helpers ----------------------------------------------------
    def fd_derivative(self, y):
        y = _c64(y)
        out = np.empty_like(y)
        _check(self.lib.fwho_fd_derivative(y.shape[0], self.dt, _d(y), _d(out)), "fd")
        return out

    def spline_moments(self, y):
        y = _c64(y)
        m = np.empty_like(y)
        _check(self.lib.fwho_natural_spline_moments(y.shape[0], self.dt, _d(y), _d(m)),
               "spline")
        return m

    def spline_eval(self, y, m, x):
        y, m, x = _c64(y), _c64(m), _c64(x)
        out = np.empty_like(x)
        _check(self.lib.fwho_spline_eval(y.shape[0], self.dt, _d(y), _d(m), x.shape[0],
                                         _d(x), _d(out)), "spline_eval")
        return out


def forward_moving(y, normals, velocities, areas, c0, rho0, dt, fields, x0, w=(0.0, 0.0, 0.0),
                   threads=0):
    """General moving surface (Eqs. pT, pL of Sec. II B): p_out [O][nt],
    t_start [O], n_valid [O].  y, normals, velocities: [nt][P][3]; areas [P];
    fields [nt][5][P] (rho', u_1..3 in the medium's frame, p'); observers start
    at x0 [O][3] and move with velocity w."""
    lib = load_oracle()
    y, n, v = _c64(y), _c64(normals), _c64(velocities)
    dS, f = _c64(areas).reshape(-1), _c64(fields)
    x = _c64(x0).reshape(-1, 3)
    ww = _c64(w).reshape(3)
    nt, P = y.shape[0], y.shape[1]
    assert n.shape == y.shape and v.shape == y.shape and f.shape == (nt, 5, P)
    O = x.shape[0]
    p_out = np.empty((O, nt))
    ts, nv = np.empty(O), np.empty(O, dtype=np.int64)
    _check(lib.fwho_forward_moving(P, nt, _d(y), _d(n), _d(v), _d(dS), float(c0), float(rho0),
                                   float(dt), _d(f), O, _d(x), _d(ww), int(threads), _d(p_out),
                                   _d(ts), nv.ctypes.data_as(_I)), "forward_moving")
    return p_out, ts, nv


def max_threads() -> int:
    return int(load_oracle().fwho_max_threads())
