"""CUDA path vs the FP64 CPU oracle, element by element (needs a GPU).

Tolerances (the accuracy bar of the two forms): rel-L2 per observer signal <= 1e-10 for the
FP64 path and <= 1e-4 for the mixed path, compared on the common prefix of
the two observer windows (N_o comes from a floor() of FP64 values that may
round differently).  Cases span several tiles with ragged tails: panel
counts that are not multiples of the 16-panel prep tile or the 64-panel set,
record lengths that are not multiples of the 128-sample chunk, one observer,
unstructured (Morton-ordered) geometry, high Mach and negative AoA.
"""
import zlib

import numpy as np
import pytest
import torch

from fwh_inputs import FlowCase, observers_circle, uv_sphere, workload
from fwh_inputs.analytic import surface_fields
from oracle import Oracle

pytestmark = pytest.mark.gpu
DEG = np.pi / 180
TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def _fwh(surf, mach, aoa, dt, prec, obs):
    from paper_2312_16263_gb300 import FWH
    return FWH(surf.centroids, surf.normals, surf.areas, mach, aoa, dt, prec, observers=obs)


def _compare(p_gpu, nv_gpu, p_ref, nv_ref, tol, label=""):
    worst = 0.0
    for o in range(p_ref.shape[0]):
        n = int(min(nv_gpu[o], nv_ref[o]))
        assert abs(int(nv_gpu[o]) - int(nv_ref[o])) <= 1, (label, o, nv_gpu[o], nv_ref[o])
        if n == 0:
            continue
        ref = p_ref[o, :n]
        den = np.linalg.norm(ref)
        err = np.linalg.norm(p_gpu[o, :n] - ref) / den if den > 0 else np.abs(p_gpu[o, :n]).max()
        worst = max(worst, err)
        # bins beyond the window are exactly zero
        assert np.all(p_gpu[o, nv_gpu[o]:] == 0.0), (label, o)
    assert worst <= tol, (label, worst)
    return worst


def _run_case(dev, surf, mach, aoa, dt, fields64, obs, prec):
    s = _fwh(surf, mach, aoa, dt, prec, obs)
    f = torch.as_tensor(fields64).to(device=dev, dtype=s.dtype).contiguous()
    p = s.forward(f).cpu().numpy()
    ts, nv = s.window(fields64.shape[0])
    s.check()
    orc = Oracle(surf.centroids, surf.normals, surf.areas, mach, aoa, dt)
    # the oracle sees exactly the values the GPU saw (float32 inputs upcast)
    p_ref, ts_ref, nv_ref = orc.forward(f.double().cpu().numpy(), obs)
    np.testing.assert_allclose(ts, ts_ref, rtol=1e-13, atol=0)
    return p, nv, p_ref, nv_ref, s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_workload1_parity(dev, prec):
    w = workload(1)
    p, nv, p_ref, nv_ref, _ = _run_case(dev, w.surface, w.mach, w.aoa, w.dt,
                                        w.fields().numpy(), w.observers, prec)
    _compare(p, nv, p_ref, nv_ref, TOL[prec], "workload1")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["ragged", "min_nt", "one_obs", "unstructured", "high_mach",
                                  "many_obs", "one_panel"])
def test_edge_cases(dev, prec, case):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    mach, aoa, dt = 0.35, -12 * DEG, 0.03
    surf = uv_sphere(1.0, 7, 11)          # 77 panels: ragged vs 16/64
    nt = 301                              # ragged vs the 128-sample chunk
    obs = observers_circle(25.0, 5) + rng.normal(size=(5, 3))
    if case == "min_nt":
        nt = 3
        obs = observers_circle(3.0, 3)
    elif case == "one_obs":
        obs = np.array([[0.0, -30.0, 2.0]])
    elif case == "unstructured":
        pts = rng.normal(size=(600, 3))
        pts /= np.linalg.norm(pts, axis=1, keepdims=True)
        from fwh_inputs.geometry import Surface
        surf = Surface(pts * 1.3, pts.copy(), rng.uniform(0.5, 1.5, 600) * 4 * np.pi * 1.69 / 600)
        nt = 700
    elif case == "high_mach":
        mach, aoa, dt = 0.9, 30 * DEG, 0.02
        nt = 513
    elif case == "many_obs":
        obs = observers_circle(40.0, 150)
        nt = 260
    elif case == "one_panel":
        from fwh_inputs.geometry import Surface
        surf = Surface(np.array([[0.2, -0.1, 0.3]]), np.array([[0.0, 0.6, 0.8]]), np.array([0.05]))
    flow = FlowCase(mach, aoa)
    f = surface_fields("monopole", surf.centroids, flow, 0.01, 2 * np.pi, dt, nt)
    f += rng.normal(size=f.shape) * 1e-4      # break symmetry, exercise all terms
    p, nv, p_ref, nv_ref, _ = _run_case(dev, surf, mach, aoa, dt, f, obs, prec)
    _compare(p, nv, p_ref, nv_ref, TOL[prec], case)


@pytest.mark.parametrize("n_phi", [11, 10])
def test_mixed_prep_block_boundaries(dev, n_phi):
    """The FP32 series of 64-sample blocks whose filters stay inside rows
    1..nt-2 come from the persistent interior kernel (derivative-series
    moments as differences of value-series moments), the rest from the
    general kernel, which filters the point-reflected series from 82 frames
    on and the odd-periodic extension of r by index arithmetic below that
    (nt = 40, 81 / 82).  Record lengths put the first interior block on and
    off (nt = 144 / 145 / 146), move the last one (209 / 210, 337) and give
    long runs of interior blocks within and across 8-block work units (600,
    1100); 77 panels take the 4-byte copy path, 80 panels the 16-byte one."""
    rng = np.random.default_rng(17 + n_phi)
    mach, aoa, dt = 0.4, 7 * DEG, 0.03
    surf = uv_sphere(1.0, 7 if n_phi == 11 else 8, n_phi)
    obs = observers_circle(6.0, 4) + rng.normal(size=(4, 3)) * 0.5
    flow = FlowCase(mach, aoa)
    for nt in (40, 81, 82, 144, 145, 146, 209, 210, 337, 600, 1100):
        f = surface_fields("dipole", surf.centroids, flow, 0.01, 2 * np.pi, dt, nt)
        f += rng.normal(size=f.shape) * 1e-4
        p, nv, p_ref, nv_ref, _ = _run_case(dev, surf, mach, aoa, dt, f, obs, "mixed")
        assert int(nv.max()) > 0, nt
        _compare(p, nv, p_ref, nv_ref, TOL["mixed"], f"blocks nt={nt}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_workload2_full_size_sampled(dev, prec):
    """Full workload 2 (32768 panels x 2048 steps x 72 observers) in the
    bench's launch configuration; the oracle checks 4 sampled observers."""
    w = workload(2)
    from paper_2312_16263_gb300 import FWH
    s = FWH.from_workload(w, prec)
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32")
    p = s.forward(f).cpu().numpy()
    s.check()
    _, nv = s.window(w.nt)
    pick = np.array([0, 18, 41, 63])
    orc = Oracle.from_workload(w)
    p_ref, _, nv_ref = orc.forward(f.double().cpu().numpy(), w.observers[pick])
    _compare(p[pick], nv[pick], p_ref, nv_ref, TOL[prec], "workload2")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_host_pointer_path_matches_device(dev, prec):
    w = workload(1, scale=0.5)
    from paper_2312_16263_gb300 import FWH
    s = FWH.from_workload(w, prec)
    f = w.fields(dtype="float64" if prec == "fp64" else "float32")
    p_host = s.forward(f.contiguous())          # host in, host out (staged)
    p_dev = s.forward(f.to(dev)).cpu()
    assert p_host.device.type == "cpu"
    assert torch.allclose(p_host, p_dev, rtol=0, atol=1e-14 * p_dev.abs().max().item())


@pytest.mark.parametrize("cfg", [0, 5, 11])
def test_host_slab_pipeline_matches_device(dev, cfg):
    """Host FP32 fields of 256 frames or more are copied in 128-frame slabs,
    each slab's series prepared once the next has landed and each two-chunk
    time segment of the scatter launched once its rows are ready (256-sample
    segments under tile shape 0, 512 under shape 5).  The result must match
    one copy followed by one prep and one scatter: exact-slab, ragged-last-
    slab and below-threshold record lengths, from pinned and pageable memory,
    with a device output too.  The series are the same bits either way; the
    shorter scatter segments split the FP32 per-bin partial sums at segment
    boundaries differently, so the outputs agree to the rounding of those
    sums: at most 1e-6 relative L2 per observer with plain FP32 window sums
    (2.9e-7 measured on a GB300) and 1e-7 with the compensated sums of shape
    11 (1.5e-8 measured); stale or missing series would be O(1)."""
    tol = 1e-7 if cfg == 11 else 1e-6
    w = workload(4)
    from paper_2312_16263_gb300 import FWH
    s = FWH.from_workload(w, "mixed")
    s.set_tile_config(cfg)
    f_all = w.fields(dtype="float32")

    def rel(p, ref):
        den = torch.linalg.norm(ref, dim=1)
        return (torch.linalg.norm(p - ref, dim=1) / torch.where(den > 0, den, 1)).max().item()

    for nt in (255, 256, 257, 383, 700, 1024):
        f = f_all[:nt].contiguous()
        p_dev = s.forward(f.to(dev)).cpu()
        assert p_dev.abs().max().item() > 0, nt
        _, nv = s.window(nt)
        for src in (f, f.pin_memory()):
            p_host = s.forward(src)
            assert p_host.device.type == "cpu"
            assert rel(p_host, p_dev) <= tol, nt
            # bins past each observer's window stay exactly zero
            for o, n in enumerate(nv):
                assert torch.all(p_host[o, int(n):] == 0), (nt, o)
        # host fields, device output: the call may return before the stream
        # is done; the stream orders the read-back
        out = torch.empty((s.O, nt), dtype=torch.float64, device=dev)
        f_pinned = f.pin_memory()
        s.forward(f_pinned, out)
        assert rel(out.cpu(), p_dev) <= tol, nt
        del f_pinned


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n_obs", [6, 80])
@pytest.mark.parametrize("npol,naz,nt", [(9, 13, 333), (8, 16, 83), (8, 16, 61)])
def test_backward_matches_oracle_adjoint(dev, prec, n_obs, npol, naz, nt):
    """Adjoint vs the oracle's FP64 adjoint.  In the mixed form, 80 observers
    make three 36-observer groups whose partial gradients are added with
    atomics (6 observers: one group, direct stores).  Two sphere meshes (117
    and 128 panels); in the FP32 adjoint prep the record ends take one
    reflection per end from 83 steps up (333 and 83) and the general
    odd-periodic extension below that (61)."""
    rng = np.random.default_rng(5)
    surf = uv_sphere(1.0, npol, naz)
    mach, aoa, dt = 0.45, 8 * DEG, 0.04
    obs = observers_circle(20.0, n_obs) + rng.normal(size=(n_obs, 3))
    f = surface_fields("dipole", surf.centroids, FlowCase(mach, aoa), 0.01, 2 * np.pi, dt, nt)
    f += rng.normal(size=f.shape) * 1e-3
    s = _fwh(surf, mach, aoa, dt, prec, obs)
    ft = torch.as_tensor(f).to(device=dev, dtype=s.dtype).contiguous()
    g_out = torch.as_tensor(rng.normal(size=(obs.shape[0], nt)), device=dev)
    g = s.backward(ft, g_out).double().cpu().numpy()
    s.check()
    orc = Oracle(surf.centroids, surf.normals, surf.areas, mach, aoa, dt)
    g_ref = orc.backward(ft.double().cpu().numpy(), obs, g_out.cpu().numpy())
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert err <= (1e-10 if prec == "fp64" else 1e-4), err


@pytest.mark.parametrize("ring", [0, 512])
@pytest.mark.parametrize("form", ["pipelined", "grid", "persistent"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_forward_matches_single(dev, prec, form, ring):
    """Three small surfaces (one record of three 512-sample segments) in one
    batched call, in every launch form, with whole records and with a
    one-segment ring (three rounds), equal to one fwh_forward call per
    surface to the rounding of the output sums.  FP64 runs the direct-load
    shape with whole records and the copy-pipeline shape with the ring."""
    from paper_2312_16263_gb300 import FWH, batch_forward
    rng = np.random.default_rng(11)
    surfs, fields, singles = [], [], []
    dtype = torch.float64 if prec == "fp64" else torch.float32
    cfg = 1 if (prec == "fp64" and ring) else -1
    for i, (npol, naz, nt, no) in enumerate([(8, 16, 200, 5), (13, 7, 131, 9), (20, 40, 1100, 3)]):
        sf = uv_sphere(1.0 + 0.3 * i, npol, naz, center=(i, 0, 0))
        obs = observers_circle(30.0, no) + rng.normal(size=(no, 3))
        s = FWH(sf.centroids, sf.normals, sf.areas, 0.3 + 0.1 * i, 0.1 * i, 0.02, prec,
                observers=obs)
        s.set_tile_config(cfg)
        f = torch.as_tensor(rng.normal(size=(nt, 5, sf.n_panels)) * 1e-3, dtype=dtype, device=dev)
        surfs.append(s)
        fields.append(f)
        singles.append(s.forward(f).clone())
    surfs[0].set_batch_options(ring, form)
    for _ in range(2):  # second call replays the captured graph
        outs = batch_forward(surfs, fields)
        for a, b in zip(outs, singles):
            torch.testing.assert_close(a, b, rtol=1e-12, atol=1e-12 * b.abs().max().item())
    surfs[0].check()


def test_batch_options_rejected(dev):
    """A negative ring length or an unknown launch form is refused with
    FWH_ERR_ARG and leaves the options as they were."""
    from paper_2312_16263_gb300 import FWH, _abi
    sf = uv_sphere(1.0, 8, 16)
    s = FWH(sf.centroids, sf.normals, sf.areas, 0.3, 0.0, 0.02, "mixed",
            observers=observers_circle(30.0, 4))
    assert s.lib.fwh_set_batch_options(s.h, -1, _abi.FWH_BATCH_GRID) == _abi.FWH_ERR_ARG
    assert s.lib.fwh_set_batch_options(s.h, 0, 3) == _abi.FWH_ERR_ARG
    assert s.lib.fwh_set_batch_options(s.h, 512, _abi.FWH_BATCH_PERSISTENT) == _abi.FWH_OK
    with pytest.raises(KeyError):
        s.set_batch_options(0, "queue")
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_tile_config_agrees(dev, prec):
    """Every forward tile configuration (direct-load and TMA-pipeline kernels)
    gives the oracle's answer; the autotuner picks one of them."""
    w = workload(1, scale=0.5)
    from paper_2312_16263_gb300 import FWH, _abi
    s = FWH.from_workload(w, prec)
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32")
    orc = Oracle.from_workload(w)
    p_ref, _, nv_ref = orc.forward(f.double().cpu().numpy(), w.observers)
    _, nv = s.window(w.nt)
    n = 0
    while True:
        try:
            s.set_tile_config(n)
        except _abi.FWHError:
            break
        out = s.forward(f).cpu().numpy()
        s.check()
        _compare(out, nv, p_ref, nv_ref, TOL[prec], f"config {n}")
        n += 1
    assert n >= 3
    chosen = s.autotune(w.nt)
    assert 0 <= chosen < n
    s.check()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nt", [1024, 1100, 513])
def test_segment_pipeline_matches_one_launch(dev, prec, nt):
    """Device fields over several 512-sample segments: the pipelined call
    (series of each segment prepared on the prep stream, the segment scattered
    as soon as they are in) equals the prep-then-one-launch call to the FP64
    rounding of the output sums (the same FP32 partial sums reach the output
    bins, in another order)."""
    from paper_2312_16263_gb300 import FWH
    w = workload(4)
    s = FWH.from_workload(w, prec)
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32", nt=nt)
    s.set_pipeline(False)
    ref = s.forward(f).clone()
    s.set_pipeline(True)
    for _ in range(2):
        p = s.forward(f)
        s.check()
        torch.testing.assert_close(p, ref, rtol=1e-12, atol=1e-13 * ref.abs().max().item())
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_empty_observer_window_gives_zeros(dev, prec):
    """A record shorter than the arrival-time spread over the surface leaves no
    valid observer bin (N_o = 0): the output is all zeros, like the oracle's."""
    surf = uv_sphere(1.0, 6, 10)
    mach, aoa, dt, nt = 0.5, 0.0, 1e-3, 40          # spread ~ 1000 samples >> nt
    obs = observers_circle(30.0, 4)
    f = np.random.default_rng(3).normal(size=(nt, 5, surf.n_panels)) * 1e-3
    p, nv, p_ref, nv_ref, _ = _run_case(dev, surf, mach, aoa, dt, f, obs, prec)
    assert np.all(nv == 0) and np.all(nv_ref == 0)
    assert np.all(p == 0.0)


def test_oversized_mixed_problem_is_refused_and_the_handle_survives(dev):
    """Mixed handles address series rows with 32-bit indices: panels x steps
    (rounded up to 256) at or above 2^32 is refused before any kernel runs, and
    the handle keeps working for a valid length afterwards."""
    import ctypes
    from paper_2312_16263_gb300 import FWH, _abi
    n = 1 << 21                                      # 2M panels on a sphere
    th = np.arccos(1 - 2 * (np.arange(n) + 0.5) / n)
    ph = np.pi * (1 + 5 ** 0.5) * np.arange(n)
    nrm = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    s = FWH(nrm * 1.0, nrm.copy(), np.full(n, 4 * np.pi / n), 0.3, 0.1, 0.02, "mixed",
            observers=np.array([[0.0, -20.0, 0.0]]))
    dummy = torch.zeros(16, device=dev)
    out = torch.zeros(2, device=dev, dtype=torch.float64)
    st = s.lib.fwh_forward(s.h, ctypes.c_void_p(dummy.data_ptr()), 2049,
                           ctypes.c_void_p(out.data_ptr()), None)
    assert st == _abi.FWH_ERR_ARG and b"2^32" in s.lib.fwh_last_error(s.h)
    nt = 8
    f = torch.zeros((nt, 5, n), dtype=torch.float32, device=dev)
    f[:, 4] = 1e-3
    p = s.forward(f)
    s.check()
    assert torch.isfinite(p).all()
    s.close()


@pytest.mark.parametrize("kahan_cfg", [10, 11])
def test_compensated_window_sums_stress(dev, kahan_cfg):
    """Long in-set sums: low Mach and a coarse step keep the arrival spread of
    a panel set small, so sets fill to their 64-panel cap and every window
    slot sums about 128 terms per set in FP32.  The plain and the compensated
    (Kahan) window sums both meet the mixed bar against the oracle; the
    compensated sums are at least as accurate and agree with the FP64 path to
    within the FP32 arithmetic of the integrands."""
    from paper_2312_16263_gb300 import FWH
    surf = uv_sphere(1.0, 64, 128)                       # 8192 panels
    mach, aoa, dt, nt = 0.1, 3 * DEG, 0.05, 700
    obs = observers_circle(60.0, 6)
    rng = np.random.default_rng(21)
    f = surface_fields("monopole", surf.centroids, FlowCase(mach, aoa), 0.01, 2 * np.pi, dt, nt)
    f += rng.normal(size=f.shape) * 2e-3                 # broadband noise: cancelling terms
    s = FWH(surf.centroids, surf.normals, surf.areas, mach, aoa, dt, "mixed", observers=obs)
    fd = torch.as_tensor(f, dtype=torch.float32, device=dev)
    orc = Oracle(surf.centroids, surf.normals, surf.areas, mach, aoa, dt)
    p_ref, _, nv_ref = orc.forward(fd.double().cpu().numpy(), obs)
    _, nv = s.window(nt)
    errs = {}
    for cfg in (0, kahan_cfg):
        s.set_tile_config(cfg)
        p = s.forward(fd).cpu().numpy()
        s.check()
        errs[cfg] = _compare(p, nv, p_ref, nv_ref, TOL["mixed"], f"config {cfg}")
    assert errs[kahan_cfg] <= 1.5 * errs[0] + 1e-9, errs
    s.close()
