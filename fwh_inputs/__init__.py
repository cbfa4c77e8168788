"""Seeded synthetic inputs for the FW-H hot path (geometry, observers, fields).

Shared by the oracle tests, the CUDA parity tests and the benchmark; holds no
FW-H arithmetic (see each module's docstring for its recipe).
"""
from .analytic import FlowCase, exact_pressure, harmonic_source, surface_fields
from .geometry import (Surface, ellipsoid, extruded_contour, observers_circle,
                       observers_fibonacci, uv_sphere)
from .workloads import Workload, batch_workloads, workload

__all__ = [
    "FlowCase", "Surface", "Workload", "batch_workloads", "ellipsoid", "exact_pressure",
    "extruded_contour", "harmonic_source", "observers_circle", "observers_fibonacci",
    "surface_fields", "uv_sphere", "workload",
]
