"""fwh_forward_moving (the general moving-surface form, Eqs. pT and pL of
Sec. II B) against the FP64 oracle, element by element (needs a GPU).

At <= 1e-10 rel-L2 per observer (FP64 on both sides; the GPU finds tau* by
Newton's method, the oracle by bisection): surfaces moving with the flow of
the wind-tunnel workloads and co-moving observers (where the library's
wind-tunnel path must agree too), spinning and translating spheres around a
monopole, ragged sizes, one observer, and a problem large enough that the
observers are split over several launches.
"""
import numpy as np
import pytest
import torch

from fwh_inputs import workload
from fwh_inputs.geometry import observers_circle, uv_sphere
from oracle.oracle import forward_moving as oracle_moving

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def _compare(p, nv, p_ref, nv_ref):
    worst = 0.0
    for o in range(p_ref.shape[0]):
        assert abs(int(nv[o]) - int(nv_ref[o])) <= 1
        n = int(min(nv[o], nv_ref[o]))
        if n == 0:
            continue
        den = np.linalg.norm(p_ref[o, :n])
        worst = max(worst, float(np.linalg.norm(p[o, :n] - p_ref[o, :n]) / den))
        assert np.all(p[o, nv[o]:] == 0.0)
    assert worst <= TOL, worst
    return worst


def _run(dev, y, n, v, dS, c0, rho0, dt, f, x0, w):
    from paper_2312_16263_gb300 import moving_forward
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    p, ts, nv = moving_forward(t(y), t(n), t(v), dS, c0, rho0, dt, t(f), x0, w)
    p_ref, ts_ref, nv_ref = oracle_moving(y, n, v, dS, c0, rho0, dt, f, x0, w)
    np.testing.assert_allclose(ts, ts_ref, rtol=1e-13)
    _compare(p.cpu().numpy(), nv, p_ref, nv_ref)
    return p, nv


def _comoving(w_):
    U = np.array([np.cos(w_.aoa), np.sin(w_.aoa), 0.0])
    nt, P = w_.nt, w_.surface.n_panels
    tau = np.arange(nt) * w_.dt
    y = w_.surface.centroids[None] - tau[:, None, None] * U
    n = np.broadcast_to(w_.surface.normals, (nt, P, 3)).copy()
    v = np.broadcast_to(-U, (nt, P, 3)).copy()
    return y, n, v, U


@pytest.mark.parametrize("idx,nt", [(1, 256), (4, 300)])
def test_comoving_surface_matches_oracle_and_wind_tunnel_path(dev, idx, nt):
    from paper_2312_16263_gb300 import FWH
    w_ = workload(idx, scale=0.5 if idx == 4 else 1.0)
    w_.nt = nt
    f = w_.fields("float64").numpy()
    y, n, v, U = _comoving(w_)
    p, nv = _run(dev, y, n, v, w_.surface.areas, 1.0 / w_.mach, 1.0, w_.dt, f, w_.observers, -U)
    s = FWH.from_workload(w_, "fp64")
    p_wt = s.forward(torch.as_tensor(f, device=dev)).cpu().numpy()
    _, nv_wt = s.window(nt)
    _compare(p.cpu().numpy(), nv, p_wt, nv_wt)
    s.close()


def _sphere(motion, n_pol, n_az, nt, dt):
    import test_oracle_moving as tom
    s = uv_sphere(1.0, n_pol, n_az)
    tau = np.arange(nt) * dt
    P = s.n_panels
    if motion == "spin":
        Om = 0.3
        c, sn = np.cos(Om * tau), np.sin(Om * tau)
        rot = np.zeros((nt, 3, 3))
        rot[:, 0, 0], rot[:, 0, 1], rot[:, 1, 0], rot[:, 1, 1], rot[:, 2, 2] = c, -sn, sn, c, 1
        y = np.einsum("tij,pj->tpi", rot, s.centroids)
        n = np.einsum("tij,pj->tpi", rot, s.normals)
        v = np.cross(np.array([0.0, 0.0, Om]), y)
    else:
        V = np.array([0.08, -0.05, 0.02])
        y = s.centroids[None] + tau[:, None, None] * V
        n = np.broadcast_to(s.normals, (nt, P, 3)).copy()
        v = np.broadcast_to(V, (nt, P, 3)).copy()
    rho, u, p = tom._monopole_fields(y, tau[:, None], 1e-4, np.pi)
    f = np.empty((nt, 5, P))
    f[:, 0], f[:, 1:4], f[:, 4] = rho, np.moveaxis(u, 2, 1), p
    return y, n, v, s.areas, f


@pytest.mark.parametrize("motion,n_pol,n_az,nt,n_obs", [("spin", 20, 40, 320, 8),
                                                        ("translate", 13, 27, 301, 5),
                                                        ("spin", 7, 9, 37, 1)])
def test_moving_spheres_match_oracle(dev, motion, n_pol, n_az, nt, n_obs):
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    y, n, v, dS, f = _sphere(motion, n_pol, n_az, nt, 0.025)
    obs = np.concatenate([observers_circle(12.0, 6), [[0.0, 0.0, 12.0], [3.0, -4.0, -11.0]]])[:n_obs]
    w = np.array([0.0, 0.0, 0.0]) if motion == "spin" else np.array([0.05, 0.0, 0.0])
    _run(dev, y, n, v, dS, 1.0, 1.0, 0.025, f, obs, w)


def test_observers_split_over_launches(dev):
    """4 x nt x P FP64 scratch columns per observer (1 GiB here) fit two
    observers in a 2 GiB budget, so the three observers take two launches."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from paper_2312_16263_gb300 import _abi
    lib = _abi.load()
    y, n, v, dS, f = _sphere("spin", 64, 128, 4096, 0.02)     # 8192 panels
    assert 3 * (4 * 4096 * 8192 * 8) > 2 << 30
    obs = observers_circle(15.0, 3)
    assert lib.fwh_set_moving_scratch(-1) == _abi.FWH_ERR_ARG
    _abi.check(lib.fwh_set_moving_scratch(2 << 30), None)
    try:
        _run(dev, y, n, v, dS, 1.0, 1.0, 0.02, f, obs, np.zeros(3))
    finally:
        _abi.check(lib.fwh_set_moving_scratch(0), None)
