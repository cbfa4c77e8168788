"""FP64 CPU oracle of the PSD post-processing of far-field signals.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU-baseline leg use
it; the product library never does.

Sec. IV C of the paper turns each observer's pressure signal into a power
spectral density by Welch's method: the signal is cut into segments with 50 %
overlap, each segment is multiplied by a Hanning window, and the squared
magnitudes of the segments' Fourier transforms are averaged.  The result is
then shifted by the span correction of Eq. PSD_corr,

    PSD_corr = PSD + 10 log10(b_exp / b_m)          (in dB),

which is the factor b_exp / b_m on the linear density.  Readings where the
text is silent (each listed in the design notes):
  * segment length L is a parameter (a power of two), step L / 2, and
    K = floor((N - L) / (L / 2)) + 1 segments of the N valid samples;
  * the Hanning window is the periodic one, w[n] = 0.5 - 0.5 cos(2 pi n / L);
  * optional removal of each segment's mean before windowing;
  * one-sided density: |X_k|^2 averaged over the segments, divided by
    fs * sum(w^2), doubled for 0 < k < L / 2;
  * dB relative to p_ref^2 when a reference pressure is given.
The steps follow that order; numpy's FFT is the transform of each segment.
"""
from __future__ import annotations

import numpy as np


def hann_periodic(L: int) -> np.ndarray:
    """The periodic Hanning window of length L (Sec. IV C)."""
    n = np.arange(L, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * n / L)


def n_segments(n: int, nperseg: int) -> int:
    """Segments of length nperseg with 50 % overlap in n samples."""
    return 0 if n < nperseg else (n - nperseg) // (nperseg // 2) + 1


def welch_psd(x, fs: float, nperseg: int, detrend: bool = True) -> np.ndarray:
    """One-sided Welch PSD [nperseg // 2 + 1] of the real signal x (Sec. IV C).

    Returns NaN everywhere when x is shorter than one segment."""
    x = np.asarray(x, dtype=np.float64)
    L = int(nperseg)
    K = n_segments(x.shape[0], L)
    if K == 0:
        return np.full(L // 2 + 1, np.nan)
    w = hann_periodic(L)
    acc = np.zeros(L // 2 + 1)
    for s in range(K):  # 50 % overlap: segment s starts at s * L / 2
        seg = x[s * (L // 2): s * (L // 2) + L]
        if detrend:
            seg = seg - seg.mean()
        X = np.fft.rfft(w * seg)
        acc += X.real ** 2 + X.imag ** 2
    P = acc / K / (fs * np.sum(w * w))
    P[1:L // 2] *= 2.0  # one-sided: the negative frequencies folded in
    return P


def psd_corr(P: np.ndarray, span_ratio: float, p_ref: float = 0.0) -> np.ndarray:
    """Span-corrected PSD (Eq. PSD_corr): linear density times b_exp / b_m, or,
    with p_ref > 0, 10 log10(PSD / p_ref^2) + 10 log10(b_exp / b_m) in dB."""
    P = np.asarray(P, dtype=np.float64)
    if p_ref > 0.0:
        return 10.0 * np.log10(P / (p_ref * p_ref)) + 10.0 * np.log10(span_ratio)
    return P * span_ratio


def observer_psd(p_out, n_valid, fs: float, nperseg: int, detrend: bool = True,
                 span_ratio: float = 1.0, p_ref: float = 0.0) -> np.ndarray:
    """PSD_corr of every row of p_out [O][nt] over its first n_valid samples."""
    p_out = np.asarray(p_out, dtype=np.float64)
    out = np.empty((p_out.shape[0], nperseg // 2 + 1))
    for o in range(p_out.shape[0]):
        n = p_out.shape[1] if n_valid is None else int(n_valid[o])
        out[o] = psd_corr(welch_psd(p_out[o, :n], fs, nperseg, detrend), span_ratio, p_ref)
    return out
