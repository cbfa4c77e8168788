"""Seeded synthetic broadband surface fields (stand-in for CFD FW-H data).

The paper's 30P30N dataset (IDDES via OpenCFD-EC, Sec. IV C) is not
available, so a sum of random convected modes with a -5/3 energy spectrum
stands in for it: mode m has frequency f_m (log-spaced up to 0.4 x Nyquist),
amplitude proportional to f_m^(-5/6), a random unit wave direction w_m,
random unit velocity polarisation q_m and random phases, and is convected at
the mean-flow speed (nondimensional 1):

    u'(y, t) = sum_m a_m q_m cos(omega_m t - k_m w_m . y + phi_m)
    p'(y, t) = sum_m a_m     cos(omega_m t - k_m w_m . y + psi_m)
    rho'     = M0^2 p'

scaled so each velocity component and p' have rms `u_rms`.  The time series
are evaluated as one real matrix product [cos, sin](omega t) x coefficients,
on any torch device.  No FW-H arithmetic lives here.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def broadband_fields(centroids: np.ndarray, mach: float, dt: float, nt: int,
                     seed: int, n_modes: int = 512, u_rms: float = 0.01,
                     device="cpu", dtype=torch.float64, t0: float = 0.0,
                     time_chunk: int = 1024) -> torch.Tensor:
    """Fields [nt][5][P] (rho', u', v', w', p') on `device` in `dtype`."""
    rng = np.random.default_rng(seed)
    P = centroids.shape[0]
    nyq = 0.5 / dt
    f_hi = 0.4 * nyq
    f_lo = max(f_hi / 1000.0, 2.0 / (nt * dt))
    f = np.exp(np.linspace(np.log(f_lo), np.log(f_hi), n_modes))
    a = f ** (-5.0 / 6.0)
    a *= math.sqrt(2.0) * u_rms / math.sqrt(np.sum(a * a))  # rms of sum = u_rms
    w = rng.normal(size=(n_modes, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    q = rng.normal(size=(n_modes, 3))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_modes)
    psi = rng.uniform(0.0, 2.0 * np.pi, n_modes)
    om = 2.0 * np.pi * f
    k = om / 1.0  # convected at the nondimensional mean-flow speed

    dev = torch.device(device)
    y = torch.as_tensor(centroids, dtype=torch.float64, device=dev)
    theta = torch.as_tensor(k[:, None], device=dev) * (torch.as_tensor(w, device=dev) @ y.T)
    # cos(om t - theta + ph) = cos(om t) cos(ph - theta) - sin(om t) sin(ph - theta)
    av = torch.as_tensor(a, device=dev)[:, None]
    cu = []
    for ph in (phi, psi):
        arg = torch.as_tensor(ph, device=dev)[:, None] - theta
        cu.append((av * torch.cos(arg), -av * torch.sin(arg)))
    qv = torch.as_tensor(q, device=dev)
    out = torch.empty((nt, 5, P), dtype=dtype, device=dev)
    omt = torch.as_tensor(om, device=dev)
    for s in range(0, nt, time_chunk):
        e = min(nt, s + time_chunk)
        t = t0 + dt * torch.arange(s, e, dtype=torch.float64, device=dev)
        C = torch.cos(t[:, None] * omt[None, :])
        S = torch.sin(t[:, None] * omt[None, :])
        # velocity components need the polarisation inside the mode sum
        for c in range(3):
            qc = qv[:, c:c + 1]
            out[s:e, 1 + c] = (C @ (qc * cu[0][0]) + S @ (qc * cu[0][1])).to(dtype)
        pp = C @ cu[1][0] + S @ cu[1][1]
        out[s:e, 4] = pp.to(dtype)
        out[s:e, 0] = (pp * mach * mach).to(dtype)
    # each velocity component: rms = u_rms * |q_c| averaged -> rescale to u_rms
    for c in range(3):
        sc = math.sqrt(float(np.sum(a * a * q[:, c] ** 2) / np.sum(a * a)))
        out[:, 1 + c] /= max(sc, 1e-12)
    return out
