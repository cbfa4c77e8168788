"""Pins of the general moving-surface oracle (Eqs. pT, pL of Sec. II B) to
things other than itself (CPU only).

* The wind-tunnel form is the general form seen from the medium's frame
  (Sec. II C): a surface moving at -U0 (with the angle of attack) through a
  medium at rest, with observers moving along with it, must give the wind-
  tunnel oracle's signals (itself pinned to the analytic convected monopole
  and dipole) to rounding: same delays (the Garrick triangle is the moving-
  observer root of Eq. tau), same integrands, same spline interpolation.
* A permeable surface is only a place where the fields are sampled: a
  sphere at rest, spinning, or translating around a stationary monopole in a
  medium at rest must reproduce the monopole's analytic far field within the
  discretisation error, and the three must agree with each other to that
  error.  A dropped Doppler factor, a wrong sign of M_r or of the
  M-dot_r term, or a mistimed retarded sample would break this.
"""
import numpy as np
import pytest

from fwh_inputs import workload
from fwh_inputs.geometry import observers_circle, uv_sphere
from oracle import Oracle
from oracle.oracle import forward_moving

DEG = np.pi / 180


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("idx", [1, 2])
def test_comoving_general_form_equals_wind_tunnel_form(idx):
    w = workload(idx, scale=0.25)
    w.nt = 160
    P, nt = w.surface.n_panels, w.nt
    f = w.fields("float64").numpy()
    p_wt, ts_wt, nv_wt = Oracle.from_workload(w).forward(f, w.observers)
    U = np.array([np.cos(w.aoa), np.sin(w.aoa), 0.0])    # nondimensional U0 = 1
    tau = np.arange(nt) * w.dt
    y = w.surface.centroids[None, :, :] - tau[:, None, None] * U   # surface at -U0
    n = np.broadcast_to(w.surface.normals, (nt, P, 3)).copy()
    v = np.broadcast_to(-U, (nt, P, 3)).copy()
    # the medium's frame: fluid velocity u' (the tunnel's U + u' minus U)
    p_mv, ts_mv, nv_mv = forward_moving(y, n, v, w.surface.areas, 1.0 / w.mach, 1.0, w.dt, f,
                                        w.observers, -U)
    np.testing.assert_allclose(ts_mv, ts_wt, rtol=1e-13)
    assert np.array_equal(nv_mv, nv_wt)
    assert nv_wt.max() > 50
    for o in range(w.observers.shape[0]):
        n_o = int(nv_wt[o])
        if n_o == 0:                       # a record shorter than this observer's spread
            assert np.all(p_mv[o] == 0.0)
            continue
        assert rel_l2(p_mv[o, :n_o], p_wt[o, :n_o]) <= 1e-10, o


def _monopole_fields(pos, t, A, om, c0=1.0, rho0=1.0):
    """Stationary monopole at the origin in a medium at rest, linear acoustics:
    phi = Re[A exp(i om (t - r/c0)) / (4 pi r)], u = grad phi, p' = -rho0 dphi/dt,
    rho' = p'/c0^2, at positions pos [..., 3] and times t [...]."""
    r = np.linalg.norm(pos, axis=-1)
    e = A * np.exp(1j * om * (t - r / c0)) / (4 * np.pi * r)
    dphidr = e * (-1.0 / r - 1j * om / c0)
    u = np.real(dphidr)[..., None] * pos / r[..., None]
    p = -rho0 * np.real(1j * om * e)
    return p / (c0 * c0), u, p


def _moving_sphere_case(motion, n_pol=20, n_az=40, nt=320, dt=0.025):
    c0, A, om = 1.0, 1e-4, 2 * np.pi * 0.5       # wavelength 2 on a unit sphere
    s = uv_sphere(1.0, n_pol, n_az)
    tau = np.arange(nt) * dt
    P = s.n_panels
    if motion == "rest":
        y = np.broadcast_to(s.centroids, (nt, P, 3)).copy()
        n = np.broadcast_to(s.normals, (nt, P, 3)).copy()
        v = np.zeros((nt, P, 3))
    elif motion == "spin":                           # about z, 0.3 c0 at the equator
        Om = 0.3
        c, sn = np.cos(Om * tau), np.sin(Om * tau)
        rot = np.zeros((nt, 3, 3))
        rot[:, 0, 0], rot[:, 0, 1], rot[:, 1, 0], rot[:, 1, 1], rot[:, 2, 2] = c, -sn, sn, c, 1
        y = np.einsum("tij,pj->tpi", rot, s.centroids)
        n = np.einsum("tij,pj->tpi", rot, s.normals)
        v = np.cross(np.array([0.0, 0.0, Om]), y)
    else:                                            # translation at 0.1 c0 along x
        V = np.array([0.1, 0.0, 0.0])
        y = s.centroids[None] + tau[:, None, None] * V
        n = np.broadcast_to(s.normals, (nt, P, 3)).copy()
        v = np.broadcast_to(V, (nt, P, 3)).copy()
    rho, u, p = _monopole_fields(y, tau[:, None], A, om, c0)
    f = np.empty((nt, 5, P))
    f[:, 0], f[:, 1:4], f[:, 4] = rho, np.moveaxis(u, 2, 1), p
    obs = np.concatenate([observers_circle(12.0, 6), [[0.0, 0.0, 12.0], [3.0, -4.0, -11.0]]])
    p_out, ts, nv = forward_moving(y, n, v, s.areas, c0, 1.0, dt, f, obs)
    exact = np.empty_like(p_out)
    for o in range(obs.shape[0]):
        tj = ts[o] + np.arange(nt) * dt
        exact[o] = _monopole_fields(obs[o][None, :].repeat(nt, 0), tj, A, om, c0)[2]
    return p_out, nv, exact


@pytest.fixture(scope="module")
def sphere_cases():
    return {m: _moving_sphere_case(m) for m in ("rest", "spin", "translate")}


@pytest.mark.parametrize("motion", ["rest", "spin", "translate"])
def test_moving_permeable_sphere_reproduces_monopole(sphere_cases, motion):
    p, nv, exact = sphere_cases[motion]
    for o in range(p.shape[0]):
        n_o = int(nv[o])
        assert n_o > 100
        assert rel_l2(p[o, :n_o], exact[o, :n_o]) <= 8e-3, (motion, o)


def test_surface_motion_does_not_change_the_far_field(sphere_cases):
    p0, nv0, _ = sphere_cases["rest"]
    for m in ("spin", "translate"):
        p, nv, exact = sphere_cases[m]
        for o in range(p.shape[0]):
            n_o = int(min(nv[o], nv0[o]))
            # windows start at different times: compare each with its exact signal
            # and the errors with each other
            e_m = rel_l2(p[o, :n_o], exact[o, :n_o])
            assert e_m <= 8e-3
    # and the spinning sphere's error converges under refinement (second order)
    coarse = _moving_sphere_case("spin", 12, 24, 320, 0.025)
    fine = _moving_sphere_case("spin", 24, 48, 320, 0.025)
    ec = max(rel_l2(coarse[0][o, :coarse[1][o]], coarse[2][o, :coarse[1][o]]) for o in range(8))
    ef = max(rel_l2(fine[0][o, :fine[1][o]], fine[2][o, :fine[1][o]]) for o in range(8))
    assert ef < 0.4 * ec, (ec, ef)
