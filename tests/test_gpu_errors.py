"""Device-side error reporting of the forward kernel's bounded waits (needs a GPU).

With fwh_set_wait_limit(h, 2000, withhold_copies=1) the copy pipeline issues
no copies, so the first stage wait of every compute warp waits for a barrier
that nothing completes and gives up after 2000 SM clocks (about a
microsecond): the kernel raises the timeout flag and returns.  Nothing faults
or hangs: no copy is in flight, every wait is bounded, and p_out is left
incomplete.  The tests check that
the timeout is reported synchronously by fwh_check, or by the next call when
the outputs stayed on the device, through the C ABI and the torch wrapper,
and that the handle computes correct results again afterwards.
"""
import ctypes

import numpy as np
import pytest
import torch

from fwh_inputs import workload
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


def _case(dev, prec):
    from paper_2312_16263_gb300 import FWH
    w = workload(1, scale=0.5)
    w.nt = 256
    s = FWH.from_workload(w, prec)
    if prec == "fp64":
        s.set_tile_config(1)  # the FP64 shape with the copy pipeline (the default loads directly)
    f = w.fields(device=dev, dtype="float64" if prec == "fp64" else "float32")
    return w, s, f


def _assert_matches_oracle(w, s, f, p):
    orc = Oracle.from_workload(w)
    p_ref, _, nv_ref = orc.forward(f.double().cpu().numpy(), w.observers)
    _, nv = s.window(w.nt)
    pc = p.cpu().numpy()
    for o in range(w.observers.shape[0]):
        n = int(min(nv[o], nv_ref[o]))
        err = np.linalg.norm(pc[o, :n] - p_ref[o, :n]) / np.linalg.norm(p_ref[o, :n])
        assert err <= TOL[s.precision], (o, err)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_timeout_reported_by_check(dev, prec):
    from paper_2312_16263_gb300 import _abi
    w, s, f = _case(dev, prec)
    out = torch.empty((s.O, w.nt), dtype=torch.float64, device=dev)
    s.set_wait_limit(2000, withhold_copies=True)
    s.forward(f, out)                         # device output: returns before the check
    st = s.lib.fwh_check(s.h, _abi_stream())
    assert st == _abi.FWH_ERR_TIMEOUT, st
    assert b"wait gave up" in s.lib.fwh_last_error(s.h)
    s.check()                                 # the flag was cleared
    s.set_wait_limit(0)                       # default bound: correct results again
    s.forward(f, out)
    s.check()
    _assert_matches_oracle(w, s, f, out)
    s.close()


def test_timeout_reported_on_next_call(dev):
    from paper_2312_16263_gb300 import _abi
    from paper_2312_16263_gb300._abi import FWHError
    w, s, f = _case(dev, "mixed")
    out = torch.empty((s.O, w.nt), dtype=torch.float64, device=dev)
    s.set_wait_limit(2000, withhold_copies=True)
    s.forward(f, out)
    torch.cuda.synchronize()                  # the flag copy has landed
    s.set_wait_limit(0)
    with pytest.raises(FWHError) as ei:       # the next call reports it and does not run
        s.forward(f, out)
    assert ei.value.status == _abi.FWH_ERR_TIMEOUT
    assert "earlier call" in str(ei.value)
    s.forward(f, out)                         # reported once; the handle works again
    s.check()
    _assert_matches_oracle(w, s, f, out)
    # host output: the call checks the flag itself before returning
    s.set_wait_limit(2000, withhold_copies=True)
    with pytest.raises(FWHError) as ei:
        s.forward(f.cpu())
    assert ei.value.status == _abi.FWH_ERR_TIMEOUT
    s.set_wait_limit(0)
    s.check()
    s.close()


def test_timeout_reaches_autograd(dev):
    from paper_2312_16263_gb300 import fwh_apply
    from paper_2312_16263_gb300._abi import FWHError
    w, s, f = _case(dev, "mixed")
    s.set_wait_limit(2000, withhold_copies=True)
    p = fwh_apply(s, f.clone().requires_grad_(True))
    torch.cuda.synchronize()
    s.set_wait_limit(0)
    with pytest.raises(FWHError):             # the backward is the next call on the handle
        (p * p).sum().backward()
    fr = f.clone().requires_grad_(True)
    p = fwh_apply(s, fr)
    (p * p).sum().backward()
    s.check()
    assert torch.isfinite(fr.grad).all()
    s.close()


def test_timeout_in_batched_call(dev):
    """Batched calls under withheld copies (every launch form, whole records
    and a ring): each compute warp gives up on its first stage (the
    persistent producer also ends its item queue), the timeout
    reaches fwh_check of the leading handle, and the same handles give correct
    results afterwards."""
    from paper_2312_16263_gb300 import FWH, _abi, batch_forward
    ws, surfs, fields = [], [], []
    for scale in (0.5, 0.25):
        w = workload(1, scale=scale)
        w.nt = 1200
        ws.append(w)
        surfs.append(FWH.from_workload(w, "mixed"))
        fields.append(w.fields(device=dev, dtype="float32"))
    singles = [sx.forward(fx).clone() for sx, fx in zip(surfs, fields)]
    for ring, form in ((0, "pipelined"), (512, "pipelined"), (0, "grid"), (0, "persistent"),
                       (512, "persistent")):
        surfs[0].set_batch_options(ring, form)
        surfs[0].set_wait_limit(2000, withhold_copies=True)
        batch_forward(surfs, fields)
        st = surfs[0].lib.fwh_check(surfs[0].h, _abi_stream())
        assert st == _abi.FWH_ERR_TIMEOUT, st
        surfs[0].set_wait_limit(0)
        outs = batch_forward(surfs, fields)
        surfs[0].check()
        for a, b in zip(outs, singles):
            torch.testing.assert_close(a, b, rtol=1e-12, atol=1e-12 * b.abs().max().item())
    _assert_matches_oracle(ws[1], surfs[1], fields[1], outs[1])
    for sx in surfs:
        sx.close()


def _abi_stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
