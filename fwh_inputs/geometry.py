"""Synthetic permeable FW-H data surfaces and observer sets.

Seeded, deterministic generators of the inputs the paper's validation cases
use (Sec. IV A-C): a UV sphere split into polar x azimuth quad subfaces
(the monopole/dipole surface, Fig. "sphere"), an ellipsoid for closed-surface
invariance checks, and a 2.5D extruded contour standing in for the 30P30N
permeable surface (one chord around the airfoil, about five chords into the
wake, spanwise length c/9, Sec. IV C).  No real 30P30N coordinates are used:
the contour is a smooth synthetic curve.

Panels follow the midpoint rule of the paper's cell-centred data
(App. A2): each subface carries a centroid y, a unit outward normal n and an
area dS.  This module holds no FW-H arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Surface:
    """Panelled surface: centroids [P,3], unit normals [P,3], areas [P] (float64)."""

    centroids: np.ndarray
    normals: np.ndarray
    areas: np.ndarray
    name: str = ""

    @property
    def n_panels(self) -> int:
        return int(self.areas.shape[0])


def uv_sphere(radius: float, n_polar: int, n_azimuth: int,
              center=(0.0, 0.0, 0.0)) -> Surface:
    """Sphere split into n_polar x n_azimuth patches (polar-major order).

    Each patch spans [theta_a, theta_b] x [phi_a, phi_b]; its area is the exact
    spherical-patch area r^2 (cos theta_a - cos theta_b) dphi, its centroid the
    point at the mid-angles on the sphere and its normal the radial unit vector
    there.
    """
    th = np.linspace(0.0, np.pi, n_polar + 1)
    ph = np.linspace(0.0, 2.0 * np.pi, n_azimuth + 1)
    thm = 0.5 * (th[:-1] + th[1:])
    phm = 0.5 * (ph[:-1] + ph[1:])
    T, F = np.meshgrid(thm, phm, indexing="ij")
    nrm = np.stack([np.sin(T) * np.cos(F), np.sin(T) * np.sin(F), np.cos(T)], -1)
    area = (radius ** 2) * (np.cos(th[:-1]) - np.cos(th[1:]))[:, None] * \
        (ph[1:] - ph[:-1])[None, :]
    c = np.asarray(center, dtype=np.float64)
    return Surface(
        centroids=(radius * nrm).reshape(-1, 3) + c,
        normals=nrm.reshape(-1, 3).copy(),
        areas=area.reshape(-1).astype(np.float64),
        name=f"sphere(r={radius},{n_polar}x{n_azimuth})",
    )


def ellipsoid(semi_axes, n_polar: int, n_azimuth: int, center=(0.0, 0.0, 0.0)) -> Surface:
    """Ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1 in polar x azimuth patches.

    Midpoint rule: centroid at the mid-parameters, area = |r_theta x r_phi|
    dtheta dphi there, normal = that cross product normalised (outward).
    """
    a, b, c = (float(v) for v in semi_axes)
    th = np.linspace(0.0, np.pi, n_polar + 1)
    ph = np.linspace(0.0, 2.0 * np.pi, n_azimuth + 1)
    thm = 0.5 * (th[:-1] + th[1:])
    phm = 0.5 * (ph[:-1] + ph[1:])
    T, F = np.meshgrid(thm, phm, indexing="ij")
    pos = np.stack([a * np.sin(T) * np.cos(F), b * np.sin(T) * np.sin(F), c * np.cos(T)], -1)
    rt = np.stack([a * np.cos(T) * np.cos(F), b * np.cos(T) * np.sin(F), -c * np.sin(T)], -1)
    rp = np.stack([-a * np.sin(T) * np.sin(F), b * np.sin(T) * np.cos(F), np.zeros_like(T)], -1)
    cr = np.cross(rt, rp)
    mag = np.linalg.norm(cr, axis=-1)
    nrm = cr / mag[..., None]
    dth = (th[1:] - th[:-1])[:, None]
    dph = (ph[1:] - ph[:-1])[None, :]
    return Surface(
        centroids=pos.reshape(-1, 3) + np.asarray(center, dtype=np.float64),
        normals=nrm.reshape(-1, 3),
        areas=(mag * dth * dph).reshape(-1),
        name=f"ellipsoid({a},{b},{c};{n_polar}x{n_azimuth})",
    )


def _airfoil_offset_curve(n: int, chord: float = 1.0, standoff: float = 1.0,
                          wake: float = 5.0) -> np.ndarray:
    """Closed smooth synthetic curve enclosing a three-element airfoil outline.

    The airfoil (slat ahead of x=0, main element on [0, c], flap behind it)
    sits inside the curve; the curve stands about `standoff` chords off the
    airfoil above, below and ahead, and runs `wake` chords downstream of the
    trailing edge.  It is a superellipse-like loop resampled to n points of
    equal arc length, traversed counter-clockwise (outward normal = right-hand
    side rotated).  Shape only: not the 30P30N geometry.
    """
    x0 = -0.15 * chord - standoff           # upstream extent (slat ahead of LE)
    x1 = chord * 1.2 + wake                 # downstream extent into the wake
    xc, ax = 0.5 * (x0 + x1), 0.5 * (x1 - x0)
    ay = 0.15 * chord + standoff             # half height
    t = np.linspace(0.0, 2.0 * np.pi, 20000, endpoint=False)
    e = 2.0 / 3.0                            # exponent < 1: boxy ends, smooth
    cx = np.sign(np.cos(t)) * np.abs(np.cos(t)) ** e
    cy = np.sign(np.sin(t)) * np.abs(np.sin(t)) ** e
    # taper the wake part slightly so the curve narrows downstream
    taper = 1.0 - 0.35 * np.clip((xc + ax * cx - chord) / (x1 - chord), 0.0, 1.0)
    pts = np.stack([xc + ax * cx, -0.05 * chord + ay * cy * taper], -1)
    seg = np.linalg.norm(np.roll(pts, -1, 0) - pts, axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    su = np.linspace(0.0, s[-1], n, endpoint=False)
    closed = np.vstack([pts, pts[:1]])
    return np.stack([np.interp(su, s, closed[:, 0]), np.interp(su, s, closed[:, 1])], -1)


def extruded_contour(n_contour: int = 1200, n_span: int = 64, span: float = 1.0 / 9.0,
                     chord: float = 1.0) -> Surface:
    """2.5D permeable surface: a closed contour in the x-y plane extruded along z.

    Panel (i, k) is contour segment i (between points i and i+1) times span
    strip k: centroid at the segment midpoint and strip mid-span, normal the
    in-plane outward normal of the segment, area segment length x strip width.
    Span ends are open (periodic spanwise direction, as in the paper's case).
    Order: span-major within contour points, i.e. panel = i * n_span + k.
    """
    pts = _airfoil_offset_curve(n_contour, chord=chord)
    nxt = np.roll(pts, -1, 0)
    mid = 0.5 * (pts + nxt)
    tang = nxt - pts
    length = np.linalg.norm(tang, axis=1)
    # counter-clockwise loop: outward normal is the tangent rotated by -90 degrees
    nrm2 = np.stack([tang[:, 1], -tang[:, 0]], -1) / length[:, None]
    dz = span / n_span
    zc = (np.arange(n_span) + 0.5) * dz - 0.5 * span
    P = n_contour * n_span
    cen = np.zeros((P, 3))
    nor = np.zeros((P, 3))
    cen[:, 0] = np.repeat(mid[:, 0], n_span)
    cen[:, 1] = np.repeat(mid[:, 1], n_span)
    cen[:, 2] = np.tile(zc, n_contour)
    nor[:, 0] = np.repeat(nrm2[:, 0], n_span)
    nor[:, 1] = np.repeat(nrm2[:, 1], n_span)
    area = np.repeat(length, n_span) * dz
    return Surface(cen, nor, area, name=f"contour({n_contour}x{n_span})")


def observers_circle(radius: float, n: int, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n observers on a circle in the x-y plane at angles 2 pi k / n, k = 0..n-1.

    With n divisible by 4 the set contains the point straight below the centre,
    (0, -r, 0), the "right below" observer of the paper's signal plots.
    """
    ang = 2.0 * np.pi * np.arange(n) / n
    c = np.asarray(center, dtype=np.float64)
    return np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n)], -1) + c


def observers_fibonacci(radius: float, n: int, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n near-uniform points on a sphere (golden-angle spiral)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - np.sqrt(5.0)) * k
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z], -1) * radius
    return pts + np.asarray(center, dtype=np.float64)
