"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks one stage of the oracle against a closed form, a textbook or
library routine, an invariant of the physics or the paper's worked cases:

* convected distance (Eqs. R_New..R2_New) vs the geometric definition solved
  by bisection, the AoA=0 forms (Eqs. R..R3) and the M0 -> 0 limit;
* finite differences (Sec. III B) exact on quadratics;
* the natural spline vs scipy's natural CubicSpline;
* integrands (Eqs. Qn_New_nd, Li_New_nd) vs the pulsation-expanded forms,
  zero for a uniform stream, and their Jacobian vs finite differences;
* the whole path vs the analytic convected monopole/dipole (Sec. IV A/B),
  second-order convergence in dt, rotation invariance of the AoA handling,
  closed-surface invariance, and the paper's dimensional cases (Tables
  monopole and dipole) through the nondimensionalisation of Sec. II D;
* the adjoint by the dot-product test and by central finite differences.
"""
import json
import os

import numpy as np
import pytest

from fwh_inputs import FlowCase, ellipsoid, observers_circle, uv_sphere
from fwh_inputs.analytic import exact_pressure, surface_fields, wave_equation_residual
from oracle import Oracle

DEG = np.pi / 180.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cases.json")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle(surf, mach, aoa, dt):
    return Oracle(surf.centroids, surf.normals, surf.areas, mach, aoa, dt)


# ---------------------------------------------------------------- geometry ----
def test_convected_distance_geometric_definition():
    """R solves |d - M0 R U| = R (sound path in the fluid frame while the
    observer drifts by -U T, T = M0 R); R-hat is the unit vector along it."""
    rng = np.random.default_rng(0)
    for mach, aoa in [(0.3, 5 * DEG), (0.6, 45 * DEG), (0.17, -20 * DEG), (0.9, 130 * DEG)]:
        o = Oracle(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.ones(1), mach, aoa, 0.1)
        d = rng.normal(size=(64, 3)) * rng.uniform(0.1, 100, size=(64, 1))
        R, Rs, Rh = o.convected_distance(d)
        U = np.array([np.cos(aoa), np.sin(aoa), 0.0])
        for i in range(d.shape[0]):
            lo, hi = 0.0, 10.0 * np.linalg.norm(d[i]) / (1 - mach)
            for _ in range(200):  # bisection on h(R) = |d - M0 R U| - R (decreasing)
                mid = 0.5 * (lo + hi)
                if np.linalg.norm(d[i] - mach * mid * U) - mid > 0:
                    lo = mid
                else:
                    hi = mid
            Rb = 0.5 * (lo + hi)
            assert abs(R[i] - Rb) <= 1e-12 * Rb
            ray = (d[i] - mach * Rb * U) / Rb
            np.testing.assert_allclose(Rh[i], ray, rtol=0, atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(Rh, axis=1), 1.0, rtol=0, atol=1e-13)


def test_convected_distance_aoa_zero_and_low_mach():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(50, 3)) * 7.0
    M0 = 0.4
    o = Oracle(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.ones(1), M0, 0.0, 0.1)
    R, Rs, Rh = o.convected_distance(d)
    b2 = 1 - M0 ** 2
    # Eqs. R, R_s, R1..R3: flow along x1
    Rs_ref = np.sqrt(d[:, 0] ** 2 + b2 * (d[:, 1] ** 2 + d[:, 2] ** 2))
    R_ref = (-M0 * d[:, 0] + Rs_ref) / b2
    np.testing.assert_allclose(Rs, Rs_ref, rtol=1e-14)
    np.testing.assert_allclose(R, R_ref, rtol=1e-14)
    np.testing.assert_allclose(Rh[:, 0], (-M0 * Rs_ref + d[:, 0]) / (b2 * R_ref), rtol=1e-13)
    np.testing.assert_allclose(Rh[:, 1:], d[:, 1:] / R_ref[:, None], rtol=1e-13)
    # M0 -> 0: R -> |d|, R-hat -> d/|d|
    o2 = Oracle(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.ones(1), 1e-9, 0.7, 0.1)
    R2, _, Rh2 = o2.convected_distance(d)
    np.testing.assert_allclose(R2, np.linalg.norm(d, axis=1), rtol=1e-8)
    np.testing.assert_allclose(Rh2, d / np.linalg.norm(d, axis=1)[:, None], atol=1e-8)


# ------------------------------------------------------- textbook numerics ----
def test_fd_exact_on_quadratics():
    o = Oracle(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.ones(1), 0.3, 0.0, 0.037)
    t = 0.037 * np.arange(40)
    y = 3.0 - 2.0 * t + 5.5 * t * t
    np.testing.assert_allclose(o.fd_derivative(y), -2.0 + 11.0 * t, rtol=0, atol=1e-11)


def test_natural_spline_matches_scipy():
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(2)
    h = 0.05
    for n in (3, 4, 7, 64):
        o = Oracle(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.ones(1), 0.3, 0.0, h)
        y = rng.normal(size=n)
        m = o.spline_moments(y)
        x = rng.uniform(0, (n - 1) * h, size=200)
        cs = CubicSpline(h * np.arange(n), y, bc_type="natural")
        np.testing.assert_allclose(o.spline_eval(y, m, x), cs(x), rtol=0, atol=1e-12)
        np.testing.assert_allclose(m, cs(h * np.arange(n), 2), rtol=0, atol=1e-9)
        # knots are interpolated; linear data are reproduced exactly
        np.testing.assert_allclose(o.spline_eval(y, m, h * np.arange(n)), y, atol=1e-13)
        lin = 2.0 + 0.5 * h * np.arange(n)
        np.testing.assert_allclose(o.spline_eval(lin, o.spline_moments(lin), x), 2.0 + 0.5 * x,
                                   atol=1e-13)


# --------------------------------------------------------------- integrands ----
def test_integrands_expanded_form_and_uniform_stream():
    rng = np.random.default_rng(3)
    P, nt, aoa = 17, 5, 7 * DEG
    n = rng.normal(size=(P, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    o = Oracle(rng.normal(size=(P, 3)), n, np.ones(P), 0.3, aoa, 0.1)
    f = rng.normal(size=(nt, 5, P)) * 0.01
    QL = o.integrands(f)
    U = np.array([np.cos(aoa), np.sin(aoa), 0.0])
    rho_p, up, pp = f[:, 0], f[:, 1:4], f[:, 4]
    un_p = np.einsum("tcp,pc->tp", up, n)
    Un = n @ U
    qn = rho_p * Un[None] + (1 + rho_p) * un_p          # pulsation-expanded Q_n
    np.testing.assert_allclose(QL[:, 0], qn, rtol=1e-12, atol=1e-17)
    for c in range(3):
        L = pp * n[None, :, c] + (1 + rho_p) * up[:, c] * (Un[None] + un_p)
        np.testing.assert_allclose(QL[:, 1 + c], L, rtol=1e-12, atol=1e-17)
    assert np.all(o.integrands(np.zeros_like(f)) == 0.0)


def test_integrands_vjp_vs_central_differences():
    rng = np.random.default_rng(4)
    P, nt = 5, 3
    n = rng.normal(size=(P, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    o = Oracle(rng.normal(size=(P, 3)), n, np.ones(P), 0.5, 0.3, 0.1)
    f = rng.normal(size=(nt, 5, P)) * 0.1
    qb = rng.normal(size=(nt, 4, P))
    g = o.integrands_vjp(f, qb)
    h = 1e-6
    for _ in range(20):
        idx = tuple(rng.integers(0, s) for s in f.shape)
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = np.sum((o.integrands(fp) - o.integrands(fm)) * qb) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-8 * max(1.0, abs(fd))


# ------------------------------------------------------------- whole path ----
def _analytic_case(kind, n_pol, n_az, r, mach, aoa, omega, dt, nt, r_obs, n_obs=8, axis=0,
                   amplitude=0.01):
    """Max over observers of the rel-L2 error vs the analytic field.

    The analytic fields solve linear acoustics while the integrands keep the
    quadratic terms of Eqs. Qn_New_nd / Li_New_nd, so the error has an O(A)
    floor (about 0.2% at A=0.01, M0=0.5); convergence checks use small A."""
    s = uv_sphere(r, n_pol, n_az)
    flow = FlowCase(mach, aoa)
    obs = observers_circle(r_obs, n_obs)
    f = surface_fields(kind, s.centroids, flow, amplitude, omega, dt, nt, axis)
    o = _oracle(s, mach, aoa, dt)
    p, ts, nv = o.forward(f, obs)
    t = ts[:, None] + dt * np.arange(nt)[None, :]
    ex = exact_pressure(kind, obs, flow, amplitude, omega, t, axis)
    return max(rel_l2(p[k, :nv[k]], ex[k, :nv[k]]) for k in range(len(nv)))


def test_analytic_generator_solves_convected_wave_equation():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(30, 3)) * 3 + 2
    for mach, aoa in [(0.3, 5 * DEG), (0.5, 10 * DEG), (0.6, 45 * DEG)]:
        res = wave_equation_residual(x, FlowCase(mach, aoa), 1.0, 2 * np.pi)
        from fwh_inputs.analytic import monopole_spatial
        scale = np.abs(monopole_spatial(x, FlowCase(mach, aoa), 1.0, 2 * np.pi).v) * 40
        assert np.all(np.abs(res) <= 1e-10 * scale)


def test_monopole_workload_1_matches_analytic():
    """Workload 1 (sphere r=1, 32x64, M0=0.3, AoA=5 deg, nt=256, dt=0.05)."""
    err = _analytic_case("monopole", 32, 64, 1.0, 0.3, 5 * DEG, 2 * np.pi, 0.05, 256, 50.0)
    assert err < 2e-2, err


def test_dipole_matches_analytic():
    """Workload-2 flow (M0=0.5, AoA=10 deg, omega=4 pi, r=1.5, r_obs=100) on a
    coarser sphere; at A=0.01 the O(A) quadratic-term floor dominates."""
    err = _analytic_case("dipole", 64, 128, 1.5, 0.5, 10 * DEG, 4 * np.pi, 0.01, 512, 100.0,
                         amplitude=1e-4)
    assert err < 5e-3, err
    err_a = _analytic_case("dipole", 64, 128, 1.5, 0.5, 10 * DEG, 4 * np.pi, 0.01, 512, 100.0)
    assert err_a < 8e-2, err_a


def test_error_floor_scales_with_amplitude():
    """The non-converging part of the error at high Mach is the quadratic
    integrand terms: it shrinks in proportion to the source amplitude A."""
    errs = [_analytic_case("monopole", 48, 96, 1.0, 0.7, 0.0, 2 * np.pi, 0.005, 2048, 50.0,
                           amplitude=a) for a in (1e-2, 1e-3)]
    assert errs[1] < 0.25 * errs[0], errs


def test_second_order_convergence_in_time():
    errs = [_analytic_case("monopole", 96, 192, 1.0, 0.3, 5 * DEG, 2 * np.pi, dt,
                           int(round(6.4 / dt)), 50.0, amplitude=1e-4)
            for dt in (0.1, 0.05, 0.025)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_zero_fields_and_linearity_in_pressure():
    s = uv_sphere(1.0, 6, 12)
    o = _oracle(s, 0.3, 0.2, 0.1)
    obs = observers_circle(20.0, 4)
    nt = 40
    p0, _, nv = o.forward(np.zeros((nt, 5, s.n_panels)), obs)
    assert np.all(p0 == 0.0)
    rng = np.random.default_rng(6)
    f1 = np.zeros((nt, 5, s.n_panels))
    f1[:, 4] = rng.normal(size=(nt, s.n_panels))
    f2 = np.zeros_like(f1)
    f2[:, 4] = rng.normal(size=(nt, s.n_panels))
    pa, _, _ = o.forward(f1, obs)
    pb, _, _ = o.forward(f2, obs)
    pc, _, _ = o.forward(2.5 * f1 - 0.5 * f2, obs)
    np.testing.assert_allclose(pc, 2.5 * pa - 0.5 * pb, rtol=1e-12, atol=1e-14)


def test_rotation_invariance_of_aoa_handling():
    """Rotating geometry and observers by -AoA about z with AoA=0 gives the same
    signals as the original AoA case (the same physical problem)."""
    rng = np.random.default_rng(7)
    s = uv_sphere(1.0, 8, 16)
    aoa, mach, dt, nt = 23 * DEG, 0.45, 0.05, 64
    obs = observers_circle(30.0, 6) + np.array([0, 0, 3.0])
    f = rng.normal(size=(nt, 5, s.n_panels)) * 1e-3
    p1, ts1, nv1 = _oracle(s, mach, aoa, dt).forward(f, obs)
    c, sn = np.cos(-aoa), np.sin(-aoa)
    Rz = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1.0]])
    f2 = f.copy()
    f2[:, 1:4] = np.einsum("ij,tjp->tip", Rz, f[:, 1:4])
    o2 = Oracle(s.centroids @ Rz.T, s.normals @ Rz.T, s.areas, mach, 0.0, dt)
    p2, ts2, nv2 = o2.forward(f2, obs @ Rz.T)
    np.testing.assert_allclose(ts1, ts2, rtol=1e-13)
    assert np.array_equal(nv1, nv2)
    np.testing.assert_allclose(p1, p2, rtol=0, atol=1e-12 * np.abs(p1).max())


def test_closed_surface_invariance():
    """Any closed permeable surface enclosing the source gives the same far field
    (Brentner & Farassat): spheres r=1, 1.5, 2 and an ellipsoid agree within
    the discretisation error, which shrinks under refinement.  Small A keeps
    the quadratic integrand terms (surface dependent) below that error."""
    flow, omega, dt, nt, A = FlowCase(0.3, 5 * DEG), 2 * np.pi, 0.02, 500, 1e-4
    obs = observers_circle(40.0, 8)

    def signal(surf):
        f = surface_fields("monopole", surf.centroids, flow, A, omega, dt, nt)
        p, ts, nv = _oracle(surf, flow.mach, flow.aoa, dt).forward(f, obs)
        return p, ts, nv

    def spread(scale):
        n1, n2 = int(24 * scale), int(48 * scale)
        runs = [signal(uv_sphere(r, n1, n2)) for r in (1.0, 1.5, 2.0)]
        runs.append(signal(ellipsoid((2.0, 1.2, 1.0), n1, n2)))
        worst = 0.0
        for k in range(obs.shape[0]):  # compare on the common observer-time range
            t0 = max(ts[k] for _, ts, _ in runs)
            t1 = min(ts[k] + dt * (nv[k] - 1) for _, ts, nv in runs)
            tc = np.linspace(t0, t1, 300)
            sig = [np.interp(tc, ts[k] + dt * np.arange(nv[k]), p[k, :nv[k]])
                   for p, ts, nv in runs]
            worst = max(worst, max(rel_l2(x, sig[0]) for x in sig[1:]))
        return worst

    coarse, fine = spread(1), spread(2)
    assert coarse < 2e-2 and fine < coarse * 0.6, (coarse, fine)


@pytest.mark.parametrize("case", ["monopole", "dipole"])
def test_paper_dimensional_cases(case):
    """Tables monopole / dipole in dimensional units, nondimensionalised with
    L_ref = 1 m, rho0, U0 = M0 c0 (Sec. II D); p* rho0 U0^2 vs the analytic p'."""
    cfg = json.load(open(GOLDEN))[case]
    c0, M0, rho0 = cfg["c0"], cfg["mach"], cfg["rho0"]
    aoa = cfg["aoa_deg"] * DEG
    U0 = M0 * c0
    omega = 2 * np.pi * cfg["f_hz"]
    nt = cfg["frames"]
    dt = cfg["duration_s"] / nt
    s = uv_sphere(cfg["sphere_radius_m"], cfg["n_polar"], cfg["n_azimuth"])
    obs = observers_circle(cfg["observer_radius_m"], cfg["n_observers"])
    flow = FlowCase(M0, aoa)
    kind = case
    axis = cfg.get("axis", 0)
    f = surface_fields(kind, s.centroids, flow, cfg["A"], omega, dt, nt, axis,
                       U0=U0, rho0=rho0)                      # dimensional fields
    Lref = 1.0
    fstar = f.copy()
    fstar[:, 0] /= rho0
    fstar[:, 1:4] /= U0
    fstar[:, 4] /= rho0 * U0 * U0
    o = Oracle(s.centroids / Lref, s.normals, s.areas / Lref ** 2, M0, aoa, dt * U0 / Lref)
    pstar, ts_star, nv = o.forward(fstar, obs / Lref)
    p = pstar * rho0 * U0 * U0
    t = (ts_star[:, None] + (dt * U0 / Lref) * np.arange(nt)[None, :]) * Lref / U0
    ex = exact_pressure(kind, obs, flow, cfg["A"], omega, t, axis, U0=U0, rho0=rho0)
    err = max(rel_l2(p[k, :nv[k]], ex[k, :nv[k]]) for k in range(len(nv)))
    assert err < 1e-2, err


# ------------------------------------------------------------------ adjoint ----
def _small_problem(seed=8):
    rng = np.random.default_rng(seed)
    s = uv_sphere(1.0, 5, 9)
    o = _oracle(s, 0.4, 12 * DEG, 0.07)
    obs = observers_circle(15.0, 3) + rng.normal(size=(3, 3))
    nt = 24
    f = rng.normal(size=(nt, 5, s.n_panels)) * 0.05
    return o, obs, f, rng


def test_adjoint_dot_product():
    o, obs, f, rng = _small_problem()
    nt = f.shape[0]
    QL = rng.normal(size=(nt, 4, o.P))
    G = rng.normal(size=(obs.shape[0], nt))
    p, _, nv = o.forward_QL(QL, obs)
    for k in range(len(nv)):
        G[k, nv[k]:] = 0.0
    lhs = np.sum(p * G)
    rhs = np.sum(QL * o.backward_QL(G, obs, nt))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.abs(p * G).sum())


def test_adjoint_vs_central_differences():
    o, obs, f, rng = _small_problem(9)

    def loss(ff):
        p, _, _ = o.forward(ff, obs)
        return float(np.sum(p * p))

    p, _, _ = o.forward(f, obs)
    g = o.backward(f, obs, 2.0 * p)
    h = 1e-6
    for _ in range(24):
        idx = tuple(int(rng.integers(0, s)) for s in f.shape)
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = (loss(fp) - loss(fm)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * np.abs(g).max() + 1e-9 * abs(fd), (idx, fd, g[idx])


def test_summation_modes_and_threads_agree():
    o, obs, f, _ = _small_problem(10)
    p1, _, _ = o.forward(f, obs, threads=1)
    p2, _, _ = o.forward(f, obs, threads=4, compensated=True)
    np.testing.assert_allclose(p1, p2, rtol=0, atol=1e-13 * np.abs(p1).max())
    # partial panel ranges sum to the whole
    pa, _, _ = o.forward(f, obs, p_range=(0, 20))
    pb, _, _ = o.forward(f, obs, p_range=(20, o.P))
    np.testing.assert_allclose(pa + pb, p1, rtol=0, atol=1e-13 * np.abs(p1).max())
