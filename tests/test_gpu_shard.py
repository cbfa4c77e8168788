"""Panel sharding through the library (Sec. III A Face partition, Sec. III B
"compute t"), three ranks emulated one after another in one process on one
GPU (needs a GPU).

Each emulated rank makes its own handle on its faces' panels; the host takes
the maximum of the ranks' R_max and the minimum of their R_min (what the
all-reduce does between processes), sets them on every handle, runs each
rank's forward pass and sums the partial signals.  The sum must equal the
oracle's unsharded result at the accuracy bar of each form, and the
library's own unsharded call.
"""
import numpy as np
import pytest
import torch

from fwh_inputs import FlowCase, observers_circle, uv_sphere
from fwh_inputs.analytic import surface_fields
from oracle import Oracle

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-4}
DEG = np.pi / 180


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_three_rank_panel_shards_sum_to_unsharded(dev, prec):
    from paper_2312_16263_gb300 import FWH
    from paper_2312_16263_gb300.shard import face_blocks, partition_faces, rank_panels
    surf = uv_sphere(1.2, 21, 40)                         # 840 panels
    mach, aoa, dt, nt = 0.45, 8 * DEG, 0.02, 300
    obs = observers_circle(40.0, 9)
    f64 = surface_fields("dipole", surf.centroids, FlowCase(mach, aoa), 0.01, 3 * np.pi, dt, nt)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    fields = torch.as_tensor(f64, dtype=dtype, device=dev)
    faces = face_blocks(surf.n_panels, 50)               # 17 faces, the last one short
    parts = partition_faces([hi - lo for lo, hi in faces], 3)
    ranks = []
    for mine in parts:
        idx = rank_panels(faces, mine)
        s = FWH(surf.centroids[idx], surf.normals[idx], surf.areas[idx], mach, aoa, dt, prec,
                observers=obs)
        ranks.append((s, idx))
    mx = np.max([s.observer_extremes()[0] for s, _ in ranks], axis=0)
    mn = np.min([s.observer_extremes()[1] for s, _ in ranks], axis=0)
    with pytest.raises(Exception):                       # must enclose the rank's own
        ranks[0][0].set_observer_extremes(mx - 1.0, mn)
    for s, _ in ranks:
        s.set_observer_extremes(mx, mn)
    p = sum(s.forward(fields[:, :, idx].contiguous()) for s, idx in ranks)
    for s, _ in ranks:
        s.check()
    full = FWH(surf.centroids, surf.normals, surf.areas, mach, aoa, dt, prec, observers=obs)
    p_full = full.forward(fields)
    ts_full, nv_full = full.window(nt)
    ts0, nv0 = ranks[0][0].window(nt)
    np.testing.assert_array_equal(nv0, nv_full)          # one common window
    np.testing.assert_allclose(ts0, ts_full, rtol=1e-15)
    orc = Oracle(surf.centroids, surf.normals, surf.areas, mach, aoa, dt)
    p_ref, _, nv_ref = orc.forward(fields.double().cpu().numpy(), obs)
    pc, pf = p.cpu().numpy(), p_full.cpu().numpy()
    for o in range(obs.shape[0]):
        n = int(min(nv0[o], nv_ref[o]))
        den = np.linalg.norm(p_ref[o, :n])
        assert np.linalg.norm(pc[o, :n] - p_ref[o, :n]) / den <= TOL[prec], o
        assert np.linalg.norm(pc[o, :n] - pf[o, :n]) / den <= TOL[prec], o
    # fwh_set_observers restores a handle's own extremes
    s0, idx0 = ranks[0]
    s0.set_observers(obs)
    mx0, _ = s0.observer_extremes()
    np.testing.assert_allclose(s0.window(nt)[0], mach * mx0, rtol=1e-15)
    for s, _ in ranks:
        s.close()
    full.close()
