"""Analytic convected monopole and dipole in a uniform flow at angle of attack.

The validation fields of Sec. IV A/B: the complex potential of a stationary
monopole in a mean flow (Eq. phi_monopole), with R and R* from the rotated
Garrick-triangle forms (Eqs. R_New, R_s_New), and the dipole as its derivative
along a chosen axis (Eq. phi_dipole, axis x2 in the paper; any axis here).
Pulsations follow Eqs. u_monopole, p_monopole, rou_monopole:
u' = grad phi,  p' = -rho0 (d/dt + U0 . grad) phi,  rho' = p' / c0^2,
with U0 = U0 (cos a, sin a, 0) (the paper's U02 is read as U0 sin a).

Everything is nondimensional (rho0 = U0 = 1, c0 = 1/M0, Sec. II D), so the
retarded phase is omega (t - M0 R).  Real parts of the complex fields are
used.  The potential separates as phi(x, t) = exp(i omega t) Phi(x): Phi, its
gradient and Hessian are evaluated once per point with a second-order forward
jet (value, gradient, Hessian) over the three coordinates, then the time
series are outer products with exp(i omega t_i).

This is the test problem's physics, not the FW-H method: nothing here
evaluates the FW-H integral.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


class Jet:
    """Second-order forward-mode jet over 3 variables: value, gradient, Hessian."""

    __slots__ = ("v", "g", "h")

    def __init__(self, v, g, h):
        self.v, self.g, self.h = v, g, h

    @staticmethod
    def variables(x: np.ndarray):
        """Independent coordinates x[..., 0..2] as three jets."""
        n = x.shape[:-1]
        out = []
        for k in range(3):
            g = np.zeros(n + (3,), dtype=x.dtype)
            g[..., k] = 1.0
            out.append(Jet(x[..., k].copy(), g, np.zeros(n + (3, 3), dtype=x.dtype)))
        return out

    def _lift(self, o):
        if isinstance(o, Jet):
            return o
        z = np.zeros_like(self.g, dtype=np.result_type(self.g, np.asarray(o)))
        return Jet(np.broadcast_to(np.asarray(o), self.v.shape) + 0 * self.v, z,
                   np.zeros_like(self.h, dtype=z.dtype))

    def __add__(self, o):
        o = self._lift(o)
        return Jet(self.v + o.v, self.g + o.g, self.h + o.h)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, -self.h)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) + (-self)

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v * o, self.g * o, self.h * o)
        gg = self.g[..., :, None] * o.g[..., None, :]
        return Jet(self.v * o.v,
                   self.g * o.v[..., None] + o.g * self.v[..., None],
                   self.h * o.v[..., None, None] + o.h * self.v[..., None, None]
                   + gg + np.swapaxes(gg, -1, -2))

    __rmul__ = __mul__

    def _apply(self, f0, f1, f2):
        """Chain rule for a scalar function with derivatives f1, f2 at self.v."""
        gg = self.g[..., :, None] * self.g[..., None, :]
        return Jet(f0, self.g * f1[..., None],
                   gg * f2[..., None, None] + self.h * f1[..., None, None])

    def sqrt(self):
        s = np.sqrt(self.v)
        return self._apply(s, 0.5 / s, -0.25 / (s * self.v))

    def exp(self):
        e = np.exp(self.v)
        return self._apply(e, e, e)

    def reciprocal(self):
        r = 1.0 / self.v
        return self._apply(r, -r * r, 2.0 * r * r * r)

    def __truediv__(self, o):
        if not isinstance(o, Jet):
            return self * (1.0 / o)
        return self * o.reciprocal()


@dataclass
class FlowCase:
    """Nondimensional mean flow: Mach number and angle of attack (radians)."""

    mach: float
    aoa: float

    @property
    def U(self) -> np.ndarray:
        return np.array([np.cos(self.aoa), np.sin(self.aoa), 0.0])


def monopole_spatial(x: np.ndarray, flow: FlowCase, amplitude: float, omega: float,
                     source=(0.0, 0.0, 0.0), c0: float | None = None) -> Jet:
    """Jet of Phi(x) = A / (4 pi R*) exp(-i omega R / c0), the spatial factor of
    Eq. phi_monopole with R, R* from Eqs. R_New, R_s_New (d = x - source).
    c0 defaults to the nondimensional sound speed 1/M0."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(source, dtype=np.float64)
    X = Jet.variables(d.astype(np.complex128))
    M0 = flow.mach
    M1, M2 = M0 * np.cos(flow.aoa), M0 * np.sin(flow.aoa)
    beta2 = 1.0 - M0 * M0
    md = X[0] * M1 + X[1] * M2
    dd = X[0] * X[0] + X[1] * X[1] + X[2] * X[2]
    Rs = (md * md + dd * beta2).sqrt()
    R = (Rs - md) * (1.0 / beta2)
    c0 = 1.0 / M0 if c0 is None else float(c0)
    phase = (R * (-1j * omega / c0)).exp()
    return phase * Rs.reciprocal() * (amplitude / (4.0 * np.pi))


@dataclass
class HarmonicField:
    """Complex spatial amplitudes of a time-harmonic potential exp(i w t) Phi(x).

    Phi, grad Phi ([N,3]) at N points; fields are Re(exp(i w t) * amp).
    """

    omega: float
    phi: np.ndarray
    grad: np.ndarray

    def pulsation_amplitudes(self, flow: FlowCase, U0: float = 1.0, rho0: float = 1.0):
        """Complex amplitudes of (rho', u', v', w', p') per point: [N, 5].

        Nondimensional by default (U0 = rho0 = 1, c0 = 1/M0); pass the
        dimensional U0 and rho0 for dimensional fields (c0 = U0 / M0)."""
        U = flow.U * U0
        p = -rho0 * (1j * self.omega * self.phi + self.grad @ U)
        c0 = U0 / flow.mach
        rho = p / (c0 * c0)
        return np.concatenate([rho[:, None], self.grad, p[:, None]], axis=1)


def harmonic_source(kind: str, x: np.ndarray, flow: FlowCase, amplitude: float,
                    omega: float, axis: int = 0, source=(0.0, 0.0, 0.0),
                    c0: float | None = None) -> HarmonicField:
    """Monopole (kind='monopole') or dipole along `axis` (kind='dipole') at x."""
    J = monopole_spatial(x, flow, amplitude, omega, source, c0)
    if kind == "monopole":
        return HarmonicField(omega, J.v, J.g)
    if kind == "dipole":
        return HarmonicField(omega, J.g[..., axis], J.h[..., axis, :])
    raise ValueError(kind)


def wave_equation_residual(x: np.ndarray, flow: FlowCase, amplitude: float, omega: float,
                           kind: str = "monopole", axis: int = 0) -> np.ndarray:
    """Residual of the convected wave equation M0^2 (i w + U.grad)^2 Phi - lap Phi
    for the monopole spatial factor (dipole: its axis derivative is also a
    solution, checked through the monopole's Hessian only).  Test helper."""
    J = monopole_spatial(x, flow, amplitude, omega)
    U = flow.U
    lap = np.trace(J.h, axis1=-2, axis2=-1)
    uHu = np.einsum("i,...ij,j->...", U, J.h, U)
    conv2 = -omega ** 2 * J.v + 2j * omega * (J.g @ U) + uHu
    return flow.mach ** 2 * conv2 - lap


def time_series(amp: np.ndarray, omega: float, t: np.ndarray) -> np.ndarray:
    """Re(exp(i omega t) amp) for amp [N, C] -> [nt, C, N] float64."""
    e = np.exp(1j * omega * np.asarray(t, dtype=np.float64))
    return np.ascontiguousarray(np.real(e[:, None, None] * amp.T[None, :, :]))


def surface_fields(kind: str, centroids: np.ndarray, flow: FlowCase, amplitude: float,
                   omega: float, dt: float, nt: int, axis: int = 0,
                   source=(0.0, 0.0, 0.0), t0: float = 0.0, U0: float = 1.0,
                   rho0: float = 1.0) -> np.ndarray:
    """Pulsation fields [nt][5][P] (rho', u', v', w', p') at panel centroids.

    Nondimensional unless a dimensional mean-flow speed U0 (and rho0) is given,
    in which case c0 = U0 / M0 and every input is in dimensional units."""
    hf = harmonic_source(kind, centroids, flow, amplitude, omega, axis, source,
                         c0=U0 / flow.mach)
    amp = hf.pulsation_amplitudes(flow, U0, rho0)
    return time_series(amp, omega, t0 + dt * np.arange(nt))


def exact_pressure(kind: str, observers: np.ndarray, flow: FlowCase, amplitude: float,
                   omega: float, t: np.ndarray, axis: int = 0,
                   source=(0.0, 0.0, 0.0), U0: float = 1.0, rho0: float = 1.0) -> np.ndarray:
    """Exact p'(x_o, t) for observers [O,3] at times t ([O, nt] or [nt])."""
    hf = harmonic_source(kind, observers, flow, amplitude, omega, axis, source,
                         c0=U0 / flow.mach)
    pa = hf.pulsation_amplitudes(flow, U0, rho0)[:, 4]
    t = np.asarray(t, dtype=np.float64)
    if t.ndim == 1:
        t = np.broadcast_to(t, (observers.shape[0], t.shape[0]))
    return np.real(np.exp(1j * omega * t) * pa[:, None])
