"""FP64 numpy oracle of the spectral losses (Sec. 4.3.1, Eq. 24-27).

TEST INFRASTRUCTURE: imported only by the tests.

STFT as the loss definitions use it: periodic Hann window of length n_fft,
hop n_fft / 4, frames centred on t = k hop (the signal is extended by
reflection by n_fft / 2 on both sides), one-sided spectrum, magnitude.

  L_log = mean over frames and bins of |log(Y + eps) - log(Yhat + eps)|  (Eq. 24)
  L_sc  = ||Y - Yhat||_F / ||Y||_F                                    (Eq. 25)
  L_sot = mean over frames of W1 between the frame spectra normalised to
          unit sum; in one dimension W1 is the L1 distance of the
          cumulative sums (Eq. 26)
"""
from __future__ import annotations

import numpy as np


def hann_periodic(n):
    k = np.arange(n)
    return 0.5 * (1.0 - np.cos(2.0 * np.pi * k / n))


def stft_mag(x, n_fft):
    """|STFT| of a 1-D signal: array [n_fft // 2 + 1][frames]."""
    x = np.asarray(x, np.float64)
    hop = n_fft // 4
    pad = n_fft // 2
    xp = np.pad(x, (pad, pad), mode="reflect")
    n_frames = 1 + (len(xp) - n_fft) // hop
    w = hann_periodic(n_fft)
    out = np.empty((n_fft // 2 + 1, n_frames))
    for k in range(n_frames):
        seg = xp[k * hop:k * hop + n_fft] * w
        out[:, k] = np.abs(np.fft.rfft(seg))
    return out


def log_stft_l1(y, target, n_fft, eps=1e-5):
    Y, T = stft_mag(y, n_fft), stft_mag(target, n_fft)
    return float(np.mean(np.abs(np.log(Y + eps) - np.log(T + eps))))


def multires_log_stft(y, target, n_ffts=(256, 1024, 4096), eps=1e-5):
    usable = [n for n in n_ffts if n // 2 < len(y)] or [min(n_ffts)]
    return sum(log_stft_l1(y, target, n, eps) for n in usable)


def spectral_convergence(y, target, n_fft=1024):
    Y, T = stft_mag(y, n_fft), stft_mag(target, n_fft)
    return float(np.linalg.norm(Y - T) / np.linalg.norm(T))


def spectral_ot(y, target, n_fft=1024, eps=1e-12):
    Y, T = stft_mag(y, n_fft), stft_mag(target, n_fft)
    Y = Y / (Y.sum(axis=0, keepdims=True) + eps)
    T = T / (T.sum(axis=0, keepdims=True) + eps)
    w1 = np.abs(np.cumsum(Y, axis=0) - np.cumsum(T, axis=0)).sum(axis=0)
    return float(w1.mean())
