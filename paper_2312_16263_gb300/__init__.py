"""GB300-native FW-H hot path of OpenCFD-FWH (arXiv 2312.16263).

The permeable-surface, nondimensional, wind-tunnel Ffowcs Williams-Hawkings
integral (thickness + loading terms of Eqs. pT_WT_nd / pL_WT_nd, Garrick
triangle with angle of attack, natural-spline interpolation onto the observer
grid) as hand-written sm_103a CUDA kernels behind the C ABI of include/fwh.h.

    from paper_2312_16263_gb300 import FWH, fwh_apply, build
    s = FWH(centroids, normals, areas, mach, aoa, dt, "mixed", observers=obs)
    p = s.forward(fields_cuda)              # [O][nt] float64

Importing the package does not load the library; the first FWH(...) does,
and fails loudly if the CUDA library is missing.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("FWH", "batch_forward", "welch_psd", "moving_forward"):
        from . import api
        return getattr(api, name)
    if name in ("fwh_apply", "FWHFunction"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)


__all__ = ["FWH", "batch_forward", "build", "fwh_apply", "FWHFunction", "welch_psd",
           "moving_forward"]
