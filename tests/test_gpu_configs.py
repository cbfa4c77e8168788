"""The remaining workload shapes through the CUDA path (needs a GPU).

* the 2.5D contour with broadband fields (76800 panels x 4096 steps x 36
  observers) at full size, the oracle checking sampled observers;
* the adjoint at the 16384-panel, 1024-step, 36-observer shape: gradients of
  loss = sum p_out^2 against FP64 central differences (h = 1e-6) of the same
  loss on 64 random (panel, time, field) entries, the finite differences taken
  with the FP64 forward path (itself pinned to the oracle at 1e-10);
* the eight uneven surfaces of the batched form, scaled down, through one
  persistent launch, against the oracle and against one call per surface.
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
def test_adjoint_against_fp64_finite_differences(dev, prec):
    from paper_2312_16263_gb300 import FWH
    w = workload(4)
    rng = np.random.default_rng(44)
    s = FWH.from_workload(w, prec)
    s64 = FWH.from_workload(w, "fp64")
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32")
    f64 = f.double()                       # the point both sides differentiate at
    p = s64.forward(f64)
    g = s.backward(f, 2.0 * p).double()    # dL/dfields, L = sum p^2
    s.check()
    nt, P = w.nt, w.surface.n_panels
    ii = rng.integers(0, nt, 64)
    cc = rng.integers(0, 5, 64)
    pp = rng.integers(0, P, 64)
    h = 1e-6
    fd = np.empty(64)
    for e in range(64):
        x = f64.clone()
        x[ii[e], cc[e], pp[e]] += h
        lp = float((s64.forward(x) ** 2).sum())
        x[ii[e], cc[e], pp[e]] -= 2 * h
        lm = float((s64.forward(x) ** 2).sum())
        fd[e] = (lp - lm) / (2 * h)
    ga = g[ii, cc, pp].cpu().numpy()
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(ga - fd).max() <= 1e-5 * scale, (np.abs(ga - fd).max(), scale)
    s.close()
    s64.close()


def _host_bytes_free():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        return 0


@pytest.mark.parametrize("prec", ["mixed"])
def test_batched_eight_surfaces_full_size(dev, prec):
    """The eight uneven surfaces at full size (524288 panels, 4096 steps, 1024
    observers each): one graph of per-segment persistent launches streaming
    the series through a two-segment ring, checked against the oracle on two
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


def test_batched_uneven_surfaces(dev):
    from paper_2312_16263_gb300 import FWH, batch_forward
    ws = batch_workloads(scale=1 / 64, nt=32768)  # 2048 steps: every window non-empty
    surfs = [FWH.from_workload(w, "mixed") for w in ws]
    fields = [w.fields(device=dev, dtype="float32") for w in ws]
    singles = [s.forward(f).clone() for s, f in zip(surfs, fields)]
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
