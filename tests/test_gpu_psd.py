"""fwh_psd (Sec. IV C, Eq. PSD_corr) against the FP64 PSD oracle (needs a GPU).

Element by element at <= 1e-10 relative (FP64 on both sides; the two FFTs
round differently): random signals of ragged lengths (an odd and an even
number of segments, a tail that no segment covers, a signal shorter than one
segment), with and without detrending, linear and dB output with the paper's
span correction, host and device buffers, every segment length from 16 to
4096; and the far-field signals of the 32768-panel dipole case over their
observer windows.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle.psd import observer_psd

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_psd.json")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build
    build()
    return torch.device("cuda:0")


def _close(a, b, tol=1e-10):
    assert np.array_equal(np.isnan(a), np.isnan(b))
    m = ~np.isnan(b)
    for r in range(b.shape[0]):
        mr = m[r]
        if not mr.any():
            continue
        err = np.abs(a[r, mr] - b[r, mr]).max() / np.abs(b[r, mr]).max()
        assert err <= tol, (r, err)


@pytest.mark.parametrize("L", [16, 64, 256, 1024, 4096])
@pytest.mark.parametrize("detrend", [True, False])
def test_psd_matches_oracle(dev, L, detrend):
    from paper_2312_16263_gb300 import welch_psd
    rng = np.random.default_rng(L + int(detrend))
    ld = 3 * L + L // 3 + 5
    nv = np.array([ld, 2 * L, L, L - 1, 3 * L // 2 + 7, ld - 1])  # K = 5, 3, 1, 0, 2, 5
    p = rng.normal(size=(nv.shape[0], ld)) + 0.2
    fs = 7.0
    ref = observer_psd(p, nv, fs, L, detrend)
    got = welch_psd(torch.as_tensor(p, device=dev), fs, L, nv, detrend).cpu().numpy()
    _close(got, ref)


def test_psd_span_correction_db_and_host_buffers(dev):
    from paper_2312_16263_gb300 import welch_psd
    g = json.load(open(GOLDEN))["span_correction"]
    ratio = g["b_exp_mm"] / g["b_m_mm"]
    rng = np.random.default_rng(11)
    p = rng.normal(size=(4, 2000)) * 1e-3
    ref = observer_psd(p, None, 50.0, 512, True, ratio, 2e-5)
    got = welch_psd(torch.as_tensor(p), 50.0, 512, None, True, ratio, 2e-5).numpy()  # host
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)  # dB: absolute
    got_d = welch_psd(torch.as_tensor(p, device=dev), 50.0, 512, None, True, ratio,
                      2e-5).cpu().numpy()
    np.testing.assert_allclose(got_d, ref, rtol=0, atol=1e-9)


def test_psd_rejects_bad_arguments(dev):
    from paper_2312_16263_gb300 import welch_psd
    from paper_2312_16263_gb300._abi import FWHError
    p = torch.zeros((2, 100), dtype=torch.float64, device=dev)
    for kw in ({"nperseg": 48}, {"nperseg": 8192}, {"nperseg": 64, "fs": -1.0}):
        with pytest.raises(FWHError):
            welch_psd(p, kw.get("fs", 1.0), kw["nperseg"])
    with pytest.raises(FWHError):
        welch_psd(p, 1.0, 64, n_valid=[100, 101])


def test_psd_of_far_field_dipole(dev):
    from fwh_inputs import workload
    from paper_2312_16263_gb300 import FWH, welch_psd
    w = workload(2)
    s = FWH.from_workload(w, "fp64")
    p = s.forward(w.fields(device=dev, dtype="float64"))
    _, nv = s.window(w.nt)
    got = welch_psd(p, 1.0 / w.dt, 512, nv).cpu().numpy()
    ref = observer_psd(p.cpu().numpy(), nv, 1.0 / w.dt, 512)
    _close(got, ref)
    # the dipole's tone (omega = 4 pi, f = 2 in these units) is the peak
    f = np.arange(257) / (512 * w.dt)
    assert np.all(np.abs(f[np.argmax(got, axis=1)] - 2.0) <= 1.0 / (512 * w.dt))
    s.close()
