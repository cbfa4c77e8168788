"""The remaining workload shapes through the CUDA path (needs a GPU).

* the 2.5D contour with broadband fields (76800 panels x 4096 steps x 36
  observers) at full size, the oracle checking sampled observers;
* the adjoint at the 16384-panel, 1024-step, 36-observer shape: gradients of
  loss = sum p_out^2 against central differences of the same loss taken
  through the oracle's forward on 64 random (panel, time, field) entries,
  each entry above a floor held to a relative bound;
* the eight uneven surfaces of the batched form, at full size and scaled
  down, whole-record and streamed through rings of time segments, against the
  oracle and against one call per surface.
"""
import os

import numpy as np
import pytest
import torch

from fwh_inputs import batch_workloads, workload
from oracle import Oracle

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def _rel_l2(p, nv, p_ref, nv_ref, idx):
    worst = 0.0
    for k, o in enumerate(idx):
        n = int(min(nv[o], nv_ref[k]))
        assert abs(int(nv[o]) - int(nv_ref[k])) <= 1
        assert n > 0, "empty observer window: the case checks nothing"
        ref = p_ref[k, :n]
        den = float(np.linalg.norm(ref))
        assert den > 0
        worst = max(worst, float(np.linalg.norm(p[o, :n] - ref)) / den)
    return worst


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_contour_broadband_full_size_sampled(dev, prec):
    from paper_2312_16263_gb300 import FWH
    w = workload(3)
    s = FWH.from_workload(w, prec)
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32")
    p = s.forward(f).cpu().numpy()
    s.check()
    _, nv = s.window(w.nt)
    pick = np.array([0, 23])
    orc = Oracle.from_workload(w)
    p_ref, _, nv_ref = orc.forward(f.double().cpu().numpy(), w.observers[pick])
    assert _rel_l2(p, nv, p_ref, nv_ref, pick) <= TOL[prec]
    s.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_adjoint_against_oracle_central_differences(dev, prec):
    """dL/dfields of L = sum p_out^2 from the CUDA adjoint against central
    differences of L taken through the oracle's forward.  The oracle's p_out
    at the fields is the point of differentiation (and, times 2, the adjoint's
    input).  For an entry (i, c, p) only subface p's share of p_out moves, so
    the two perturbed losses are L(f +- h e) = sum (a + d+-)^2 with
    a = p_out - d(f) and d the oracle's forward restricted to subface p
    (integrands of that subface, the window of the whole surface); their
    difference is formed as sum (d+ - d-)(2a + d+ + d-) so that it does not
    cancel.  The integrands are cubic in the pulsations, so the central
    difference is off by O(h^2) relative: h = 1e-4 x the component's RMS
    balances that against rounding (about 4e-10 relative on the oracle's
    own adjoint).  Every entry whose derivative is at least 1e-3 of
    the largest is held to a relative bound; the rest to that bound times
    the floor."""
    from paper_2312_16263_gb300 import FWH
    w = workload(4)
    rng = np.random.default_rng(44)
    s = FWH.from_workload(w, prec)
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32")
    f64 = f.double().cpu().numpy()
    orc = Oracle.from_workload(w)
    obs = w.observers
    p_ref, _, nv = orc.forward(f64, obs)
    g = s.backward(f, torch.from_numpy(2.0 * p_ref).to(dev)).double().cpu().numpy()
    s.check()
    s.close()
    nt, P = w.nt, w.surface.n_panels
    m = 64
    ii = rng.integers(0, nt, m)
    cc = rng.integers(0, 5, m)
    pp = rng.integers(0, P, m)
    rms = np.sqrt((f64 ** 2).mean(axis=(0, 2)))
    srf = w.surface
    zero = np.zeros((nt, 4, P))
    fd = np.empty(m)

    def share(p, fp):
        one = Oracle(srf.centroids[p:p + 1], srf.normals[p:p + 1], srf.areas[p:p + 1],
                     w.mach, w.aoa, w.dt)
        zero[:, :, p] = one.integrands(fp)[:, :, 0]
        d = orc.forward_QL(zero, obs, p_range=(p, p + 1))[0]
        zero[:, :, p] = 0.0
        return d

    for e in range(m):
        i, c, p = int(ii[e]), int(cc[e]), int(pp[e])
        h = 1e-4 * rms[c]
        fp = f64[:, :, p:p + 1].copy()
        a = p_ref - share(p, fp)
        fp[i, c, 0] += h
        dp = share(p, fp)
        fp[i, c, 0] -= 2 * h
        dm = share(p, fp)
        fd[e] = float(((dp - dm) * (2 * a + dp + dm)).sum()) / (2 * h)
    ga = g[ii, cc, pp]
    scale = np.abs(fd).max()
    assert scale > 0
    floor = 1e-3 * scale
    big = np.abs(fd) >= floor
    assert big.sum() >= 16, big.sum()
    tol = 1e-8 if prec == "fp64" else 1e-4
    rel = np.abs(ga - fd)[big] / np.abs(fd)[big]
    print(f"[adjoint vs oracle differences, {prec}] {int(big.sum())} entries, "
          f"relative error max {rel.max():.3e}, median {np.median(rel):.3e}")
    assert rel.max() <= tol, (rel.max(), np.sort(rel)[-4:])
    assert np.abs(ga - fd)[~big].max(initial=0.0) <= tol * floor


def _host_bytes_free():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        return 0


@pytest.mark.parametrize("prec", ["mixed"])
def test_batched_eight_surfaces_full_size(dev, prec):
    """The eight uneven surfaces at full size (524288 panels, 4096 steps, 1024
    observers each): whole records in the pipelined form; the same streamed
    through a ring of two 512-sample segments (four rounds), as one grid and
    as the persistent work-queue kernel, each equal to the first to the
    rounding of the output sums; the first checked against the oracle on two
    observers of every surface (rel-L2 per observer at the mixed bar) and
    against one fwh_forward call per surface."""
    from paper_2312_16263_gb300 import FWH, batch_forward
    ws = batch_workloads()
    assert sum(w.surface.n_panels for w in ws) == 524288
    surfs = [FWH.from_workload(w, prec) for w in ws]
    fields = [w.fields(device=dev, dtype="float32") for w in ws]
    outs = batch_forward(surfs, fields)
    outs = batch_forward(surfs, fields)      # the replayed graph
    surfs[0].check()
    for ring, form in ((1024, "pipelined"), (0, "grid"), (0, "persistent")):
        surfs[0].set_batch_options(ring, form)
        other = batch_forward(surfs, fields)
        surfs[0].check()
        for a, b in zip(other, outs):
            torch.testing.assert_close(a, b, rtol=1e-12, atol=1e-12 * b.abs().max().item())
        del other
    free = _host_bytes_free()
    for w, s, f, p in zip(ws, surfs, fields, outs):
        _, nv = s.window(w.nt)
        pick = np.array([0, w.observers.shape[0] // 2])
        # host FP64 fields and the oracle's integrand array: 72 bytes per panel-step
        need = 72 * w.surface.n_panels * w.nt
        if free and need > 0.5 * free:
            pytest.skip(f"host memory: the oracle on {w.name} needs {need / 1e9:.0f} GB")
        orc = Oracle.from_workload(w)
        p_ref, _, nv_ref = orc.forward(f.double().cpu().numpy(), w.observers[pick])
        assert _rel_l2(p.cpu().numpy(), nv, p_ref, nv_ref, pick) <= TOL[prec], w.name
        single = s.forward(f)
        torch.testing.assert_close(p, single, rtol=1e-12, atol=1e-12 * single.abs().max().item())
        s.close()   # frees the whole-record series before the next surface's call
    del outs


@pytest.mark.parametrize("ring,form", [(0, "pipelined"), (512, "pipelined"),
                                       (1536, "pipelined"), (0, "grid"), (1536, "grid"),
                                       (0, "persistent"), (1536, "persistent")])
def test_batched_uneven_surfaces(dev, ring, form):
    """The eight surfaces at 1/64 scale (2048 steps, four 512-sample
    segments): whole records in one launch, a one-segment ring (four rounds)
    and a three-segment ring (a full round and a one-segment round), in each
    launch form, each against one fwh_forward call per surface and the
    oracle."""
    from paper_2312_16263_gb300 import FWH, batch_forward
    ws = batch_workloads(scale=1 / 64, nt=32768)  # 2048 steps: every window non-empty
    surfs = [FWH.from_workload(w, "mixed") for w in ws]
    fields = [w.fields(device=dev, dtype="float32") for w in ws]
    singles = [s.forward(f).clone() for s, f in zip(surfs, fields)]
    surfs[0].set_batch_options(ring, form)
    for _ in range(2):  # the second call replays the captured graph
        outs = batch_forward(surfs, fields)
        for a, b in zip(outs, singles):
            torch.testing.assert_close(a, b, rtol=1e-12, atol=1e-12 * b.abs().max().item())
    surfs[0].check()
    for w, s, f, p in zip(ws, surfs, fields, outs):
        _, nv = s.window(w.nt)
        pick = np.array([0, w.observers.shape[0] // 2])
        orc = Oracle.from_workload(w)
        p_ref, _, nv_ref = orc.forward(f.double().cpu().numpy(), w.observers[pick])
        assert _rel_l2(p.cpu().numpy(), nv, p_ref, nv_ref, pick) <= TOL["mixed"], w.name
    for s in surfs:
        s.close()
