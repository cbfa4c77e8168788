"""Pins of the PSD oracle (oracle/psd.py) to things other than itself (CPU only).

The post-processing of Sec. IV C: Welch's method with 50 % overlap and a
Hanning window, then the span correction of Eq. PSD_corr.

* scipy.signal.welch (an independent implementation) with the same window,
  overlap, detrending and one-sided density scaling;
* Parseval's theorem on one segment (the density integrates to the windowed
  signal's power);
* a tone at a bin frequency integrates to A^2 / 2;
* the Hanning window equals scipy's periodic 'hann';
* the span correction with the paper's b_exp = 650 mm and b_m = 50.8 mm shifts
  the spectrum by 10 log10(650 / 50.8) = 11.07 dB.
"""
import json
import os

import numpy as np
import pytest

from oracle.psd import hann_periodic, n_segments, observer_psd, psd_corr, welch_psd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_psd.json")


@pytest.mark.parametrize("n,L", [(1024, 256), (1000, 128), (4096, 1024), (300, 64), (257, 256)])
@pytest.mark.parametrize("detrend", [True, False])
def test_welch_matches_scipy(n, L, detrend):
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(n + L)
    x = rng.normal(size=n) + 0.3 * np.sin(0.05 * np.arange(n)) + 0.7
    fs = 97.5
    f, P_ref = sig.welch(x, fs=fs, window="hann", nperseg=L, noverlap=L // 2,
                         detrend="constant" if detrend else False, scaling="density",
                         return_onesided=True)
    P = welch_psd(x, fs, L, detrend)
    np.testing.assert_allclose(P, P_ref, rtol=1e-12, atol=1e-14 * P_ref.max())
    assert np.allclose(f, np.arange(L // 2 + 1) * fs / L)


def test_hann_is_scipy_periodic_hann():
    sig = pytest.importorskip("scipy.signal")
    for L in (16, 128, 4096):
        np.testing.assert_allclose(hann_periodic(L), sig.get_window("hann", L), atol=1e-15)


def test_parseval_one_segment():
    rng = np.random.default_rng(3)
    L, fs = 512, 10.0
    x = rng.normal(size=L)
    P = welch_psd(x, fs, L, detrend=False)
    w = hann_periodic(L)
    power = np.sum((w * x) ** 2) / np.sum(w * w)
    assert abs(np.sum(P) * fs / L - power) <= 1e-12 * power


@pytest.mark.parametrize("k,A", [(5, 1.0), (37, 0.25), (100, 3.0)])
def test_tone_at_bin_integrates_to_half_square_amplitude(k, A):
    L, fs = 256, 1.0
    n = 8 * L
    t = np.arange(n)
    x = A * np.cos(2 * np.pi * k * t / L + 0.3)
    P = welch_psd(x, fs, L, detrend=True)
    assert abs(np.sum(P) * fs / L - A * A / 2) <= 1e-12 * A * A
    assert np.argmax(P) == k


def test_segment_count_and_short_signal():
    assert n_segments(1024, 256) == 7
    assert n_segments(1000, 128) == 14
    assert n_segments(255, 256) == 0
    assert np.all(np.isnan(welch_psd(np.ones(100), 1.0, 128)))


def test_span_correction_paper_values():
    g = json.load(open(GOLDEN))["span_correction"]
    ratio = g["b_exp_mm"] / g["b_m_mm"]
    rng = np.random.default_rng(5)
    P = welch_psd(rng.normal(size=2048), 2.0, 256)
    shift = psd_corr(P, ratio, p_ref=2e-5) - psd_corr(P, 1.0, p_ref=2e-5)
    np.testing.assert_allclose(shift, 11.0705, atol=5e-5)
    np.testing.assert_allclose(psd_corr(P, ratio), P * 650.0 / 50.8, rtol=1e-15)


def test_observer_psd_uses_each_window():
    rng = np.random.default_rng(9)
    p = rng.normal(size=(3, 600))
    nv = np.array([600, 400, 100])
    out = observer_psd(p, nv, 4.0, 128, True, 2.0, 0.0)
    np.testing.assert_allclose(out[1], 2.0 * welch_psd(p[1, :400], 4.0, 128), rtol=1e-15)
    assert np.all(np.isnan(out[2]))
