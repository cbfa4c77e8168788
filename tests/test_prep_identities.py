"""The exact identities the FP32 series prep of the CUDA path rests on,
checked on the CPU against the oracle's natural-spline solve (Sec. III B,
"interp pressure signal") and its time differences (central inside, one-sided
3-point at the record ends).

* The moment solve m = S r (tridiag(1, 4, 1) m = r, m_0 = m_{N-1} = 0,
  r_k = 6 (F_{k+1} - 2 F_k + F_{k-1}) / dt^2) equals, on the odd-periodic
  extension of r, the factorised Toeplitz inverse: a causal recursion
  y_k = r_k + rho y_{k-1} and an anti-causal one x_k = y_k + rho x_{k+1},
  m_k = -rho x_k, rho = sqrt 3 - 2.  Started H samples outside a block, the
  recursions err by O(|rho|^H).
* The odd-periodic extension of r is the second difference of F
  point-reflected about its end values, F(-k) = 2 F(0) - F(k),
  F(N - 1 + k) = 2 F(N - 1) - F(N - 1 - k).
* Away from the ends, the moment solve and the central difference commute:
  the moments of the derivative series are the central differences of the
  moments of the value series, up to terms that decay as |rho|^distance.
"""
import numpy as np
import pytest

from oracle import Oracle

RHO = np.sqrt(3.0) - 2.0
H = 16              # samples each recursion starts outside its block
TRUNC = RHO ** 16   # the truncation those 16 samples leave (7e-10)


def _oracle(dt):
    return Oracle(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.ones(1), 0.3, 0.0, dt)


def _series(n, dt, seed):
    """Smooth band-limited signal plus noise, like an integrand history."""
    rng = np.random.default_rng(seed)
    t = dt * np.arange(n)
    y = np.zeros(n)
    for _ in range(5):
        w = rng.uniform(0.5, 12.0)
        y += rng.normal() * np.sin(w * t + rng.uniform(0, 2 * np.pi))
    return y + 1e-2 * rng.normal(size=n)


def _reflected(F, kk):
    n = len(F)
    if kk < 0:
        return 2.0 * F[0] - F[-kk]
    if kk > n - 1:
        return 2.0 * F[n - 1] - F[2 * (n - 1) - kk]
    return F[kk]


def _blockwise_moments(F, dt, block=64, half=32):
    """Block-local recursive filtering of the point-reflected series, one
    32-sample half block at a time, each recursion started H samples
    outside it (the record-end path of the FP32 prep)."""
    n = len(F)
    s6 = 6.0 / (dt * dt)
    m = np.zeros(n)
    for ks in range(0, n, half):
        k0 = ks - H
        y = []
        yy = 0.0
        for k in range(k0, ks + half + H):
            r = s6 * (_reflected(F, k + 1) - 2.0 * _reflected(F, k) + _reflected(F, k - 1))
            yy = r + RHO * yy
            if k >= ks:
                y.append(yy)
        xx = 0.0
        for t in range(len(y) - 1, -1, -1):
            xx = y[t] + RHO * xx
            if t < half and ks + t < n:
                m[ks + t] = -RHO * xx
    return m


@pytest.mark.parametrize("n", [82, 97, 145, 300])
def test_point_reflection_is_the_odd_periodic_extension(n):
    dt = 0.03
    F = _series(n, dt, n)
    r = lambda k: (_reflected(F, k + 1) - 2.0 * _reflected(F, k) + _reflected(F, k - 1))
    scale = np.abs(F).max()
    assert abs(r(0)) <= 1e-14 * scale and abs(r(n - 1)) <= 1e-14 * scale
    for k in range(1, n - 1):
        assert abs(r(-k) + r(k)) <= 1e-13 * scale, k
        assert abs(r(n - 1 + k) + r(n - 1 - k)) <= 1e-13 * scale, k


@pytest.mark.parametrize("n", [82, 100, 211, 640])
def test_blockwise_filters_on_reflected_series_match_natural_spline(n):
    """Value and derivative series alike: the blockwise filters reproduce the
    dense natural-spline solve to |rho|^16 (7e-10) of the moments' size."""
    dt = 0.02
    o = _oracle(dt)
    for F in (_series(n, dt, 7 * n), o.fd_derivative(_series(n, dt, 7 * n))):
        m_ref = o.spline_moments(F)
        m = _blockwise_moments(F, dt)
        assert np.abs(m - m_ref).max() <= 5.0 * abs(TRUNC) * np.abs(m_ref).max()


def test_derivative_moments_are_differences_of_value_moments_inside():
    """m(D1 B) vs D1 m(B): equal up to |rho|^distance from the ends, far
    below FP32 rounding on every sample the interior kernel covers (blocks
    with c0 >= 64 and c0 + 64 + H + 1 <= N, so at least 17 samples from
    either end), and clearly different next to the ends (where the
    record-end path filters the derivative series itself)."""
    n, dt = 700, 0.025
    o = _oracle(dt)
    B = _series(n, dt, 3)
    md = o.spline_moments(o.fd_derivative(B))
    mv = o.spline_moments(B)
    alt = np.zeros(n)
    alt[1:-1] = (mv[2:] - mv[:-2]) / (2.0 * dt)
    scale = np.abs(md).max()
    dist = np.minimum(np.arange(n), n - 1 - np.arange(n))
    inside = dist >= H + 1
    err = np.abs(md - alt)
    bound = 50.0 * np.abs(RHO) ** dist * scale + 1e-11 * scale
    assert np.all(err[inside] <= bound[inside])
    assert err[inside].max() <= 1e-8 * scale
    assert err[1] >= 1e-6 * scale   # the identity does not hold at the ends


def test_interior_block_formulation_matches_derivative_series_moments():
    """The interior kernel's arithmetic, in FP64: one 64-sample block per
    (panel, integrand), the value series filtered from H + 1 samples before
    the block to H after it, derivative moments as central differences of
    the value moments, derivative series as central differences of B."""
    n, dt = 520, 0.02
    o = _oracle(dt)
    B = _series(n, dt, 11)
    s6 = 6.0 / (dt * dt)
    md_ref = o.spline_moments(o.fd_derivative(B))
    mv_ref = o.spline_moments(B)
    C = 64
    for c0 in range(64, n, C):
        if c0 + C + H + 1 > n:
            break
        y = {}
        yy = 0.0
        for k in range(c0 - 1 - H, c0 + C + H):
            yy = s6 * (B[k + 1] - 2.0 * B[k] + B[k - 1]) + RHO * yy
            if k >= c0 - 1:
                y[k] = yy
        m = {}
        xx = 0.0
        for k in range(c0 + C + H - 1, c0 - 2, -1):
            xx = y[k] + RHO * xx
            m[k] = -RHO * xx
        for k in range(c0, c0 + C):
            assert abs(m[k] - mv_ref[k]) <= 5.0 * abs(TRUNC) * np.abs(mv_ref).max()
            mdk = (m[k + 1] - m[k - 1]) / (2.0 * dt)
            assert abs(mdk - md_ref[k]) <= 20.0 * abs(TRUNC / RHO) * np.abs(md_ref).max(), k
