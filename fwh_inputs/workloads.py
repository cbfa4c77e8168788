"""The five synthetic workloads of the FW-H hot path, with their recipes.

Each workload mirrors the shape of one of the paper's cases (Sec. IV):
a panelled permeable surface, pulsation fields on it, a mean flow at AoA,
a source-time step and an observer set.  Sizes:

  1  sphere r=1, 32x64 = 2048 panels; analytic convected monopole
     (A=0.01, omega=2 pi), M0=0.3, AoA=5 deg; nt=256, dt=0.05;
     8 observers on an r=50 circle in the x-y plane.
  2  sphere r=1.5, 128x256 = 32768 panels; analytic x1-axis dipole
     (A=0.01, omega=4 pi), M0=0.5, AoA=10 deg; nt=2048, dt=0.01;
     72 observers every 5 deg on an r=100 circle.
  3  extruded synthetic contour, 1200 x 64 = 76800 panels; FP32 broadband
     fields (512 modes, -5/3 spectrum, seed 3), M0=0.17, AoA=5.5 deg;
     nt=4096, dt=1.264e-3; 36 observers on an r=10 circle.
  4  sphere r=1.5, 64x256 = 16384 panels; workload-2 dipole fields;
     nt=1024, dt=0.01; 36 observers every 10 deg on an r=100 circle.
  5  eight uneven surfaces (spheres and extruded contours, 16384..262144
     panels, 524288 in total), broadband FP32 fields (seed 100+s),
     nt=4096; 1024 observers per surface on a Fibonacci sphere r=100.

The spectrum of the broadband stand-in, its seeds and the observer recipes
are the same on both sides of every comparison: the oracle and the CUDA path
receive identical arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .analytic import FlowCase, exact_pressure, surface_fields
from .geometry import (Surface, extruded_contour, observers_circle,
                       observers_fibonacci, uv_sphere)

DEG = np.pi / 180.0


@dataclass
class Workload:
    name: str
    surface: Surface
    mach: float
    aoa: float
    dt: float
    nt: int
    observers: np.ndarray
    fields_kind: str                 # 'monopole' | 'dipole' | 'broadband'
    amplitude: float = 0.0
    omega: float = 0.0
    axis: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def flow(self) -> FlowCase:
        return FlowCase(self.mach, self.aoa)

    @property
    def evals(self) -> int:
        return self.surface.n_panels * self.nt * self.observers.shape[0]

    def fields(self, dtype="float64", device="cpu", nt=None):
        """Pulsation fields [nt][5][P] as a torch tensor (float64 or float32)."""
        import torch
        nt = self.nt if nt is None else nt
        tdt = torch.float64 if dtype in ("float64", torch.float64) else torch.float32
        if self.fields_kind in ("monopole", "dipole"):
            f = surface_fields(self.fields_kind, self.surface.centroids, self.flow,
                               self.amplitude, self.omega, self.dt, nt, self.axis)
            return torch.as_tensor(f, dtype=tdt, device=device).contiguous()
        from .broadband import broadband_fields
        return broadband_fields(self.surface.centroids, self.mach, self.dt, nt,
                                self.seed, device=device, dtype=tdt)

    def exact(self, t_obs: np.ndarray) -> np.ndarray:
        """Exact far-field p' at the observers (analytic workloads only)."""
        return exact_pressure(self.fields_kind, self.observers, self.flow,
                              self.amplitude, self.omega, t_obs, self.axis)


def workload(idx: int, scale: float = 1.0) -> Workload:
    """Workload `idx` (1..4).  scale < 1 shrinks panels and time for quick runs."""
    def s(n, m=1):
        return max(m, int(round(n * scale)))
    if idx == 1:
        return Workload("sphere-monopole-2048x256x8", uv_sphere(1.0, s(32, 4), s(64, 8)),
                        0.3, 5 * DEG, 0.05, s(256, 16), observers_circle(50.0, 8),
                        "monopole", amplitude=0.01, omega=2 * np.pi, seed=1)
    if idx == 2:
        return Workload("sphere-dipole-32768x2048x72", uv_sphere(1.5, s(128, 4), s(256, 8)),
                        0.5, 10 * DEG, 0.01, s(2048, 16), observers_circle(100.0, 72),
                        "dipole", amplitude=0.01, omega=4 * np.pi, axis=0, seed=2)
    if idx == 3:
        return Workload("contour-broadband-76800x4096x36",
                        extruded_contour(s(1200, 16), s(64, 4)),
                        0.17, 5.5 * DEG, 1.264e-3, s(4096, 16), observers_circle(10.0, 36),
                        "broadband", seed=3)
    if idx == 4:
        return Workload("sphere-dipole-16384x1024x36", uv_sphere(1.5, s(64, 4), s(256, 8)),
                        0.5, 10 * DEG, 0.01, s(1024, 16), observers_circle(100.0, 36),
                        "dipole", amplitude=0.01, omega=4 * np.pi, axis=0, seed=4)
    raise ValueError(idx)


BATCH_PANELS = (262144, 65536, 65536, 32768, 32768, 24576, 24576, 16384)


def batch_workloads(scale: float = 1.0, nt: int = 4096, n_obs: int = 1024):
    """Workload 5: eight uneven surfaces (even index sphere, odd index contour)."""
    out = []
    for i, P in enumerate(BATCH_PANELS):
        Ps = max(64, int(round(P * scale)))
        if i % 2 == 0:
            # a polar x azimuth grid of exactly Ps panels, azimuth about twice polar
            divs = [d for d in range(4, Ps // 8 + 1) if Ps % d == 0]
            n_pol = min(divs, key=lambda d: (abs(d - np.sqrt(Ps / 2)), d))
            n_az = Ps // n_pol
            surf = uv_sphere(1.0 + 0.25 * i, n_pol, n_az, center=(3.0 * i, 0.0, 0.0))
            mach, aoa, dt = 0.5, 10 * DEG, 0.01
        else:
            n_span = 64 if Ps >= 64 * 64 else 8
            surf = extruded_contour(max(16, Ps // n_span), n_span)
            surf.centroids = surf.centroids + np.array([3.0 * i, 0.0, 0.0])
            mach, aoa, dt = 0.17, 5.5 * DEG, 1.264e-3
        c = surf.centroids.mean(axis=0)
        obs = observers_fibonacci(100.0, max(4, int(round(n_obs * min(1.0, scale * 4)))), c)
        out.append(Workload(f"batch{i}-{surf.n_panels}", surf, mach, aoa, dt,
                            max(16, int(round(nt * min(1.0, scale * 4)))), obs,
                            "broadband", seed=100 + i))
    return out
