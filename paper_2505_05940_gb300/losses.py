"""Spectral losses of Sec. 4.3.1, Eq. 24-27 (user side, PyTorch ops).

    L_log = || log(Y + eps) - log(Yhat + eps) ||_1      (mean over bins, Eq. 24)
    L_sc  = || Y - Yhat ||_F / || Y ||_F                 (Eq. 25)
    L_sot = 1/N sum_frames W1(Y_i, Yhat_i)               (Eq. 26, normalised frames)

with Y = |STFT(x)| (Hann window, hop n_fft / 4).  The multi-resolution
variant sums L_log over several FFT sizes.  These run on the autograd graph
of the simulator's output; their gradient dL/dy is what the adjoint kernels
consume.
"""
from __future__ import annotations

import torch


def stft_mag(x, n_fft):
    win = torch.hann_window(n_fft, device=x.device, dtype=x.dtype)
    X = torch.stft(x, n_fft=n_fft, hop_length=n_fft // 4, win_length=n_fft, window=win,
                   center=True, return_complex=True)
    return X.abs()


def log_stft_l1(y, target, n_fft, eps=1e-5):
    Y = stft_mag(y, n_fft)
    T = stft_mag(target, n_fft)
    return (torch.log(Y + eps) - torch.log(T + eps)).abs().mean(dim=(-2, -1))


def multires_log_stft(y, target, n_ffts=(256, 1024, 4096), eps=1e-5):
    """Per-instance sum over resolutions of the mean log-magnitude L1 (Eq. 24).
    Resolutions longer than half the signal are skipped (reflect padding)."""
    usable = [n for n in n_ffts if n // 2 < y.shape[-1]] or [min(n_ffts)]
    return sum(log_stft_l1(y, target, n, eps) for n in usable)


def spectral_convergence(y, target, n_fft=1024):
    Y = stft_mag(y, n_fft)
    T = stft_mag(target, n_fft)
    return torch.linalg.vector_norm(Y - T, dim=(-2, -1)) / torch.linalg.vector_norm(T, dim=(-2, -1))


def spectral_ot(y, target, n_fft=1024, eps=1e-12):
    """Mean over frames of the 1-D Wasserstein-1 distance between the
    normalised magnitude spectra (difference of cumulative distributions)."""
    Y = stft_mag(y, n_fft)
    T = stft_mag(target, n_fft)
    Y = Y / (Y.sum(dim=-2, keepdim=True) + eps)
    T = T / (T.sum(dim=-2, keepdim=True) + eps)
    w1 = (torch.cumsum(Y, dim=-2) - torch.cumsum(T, dim=-2)).abs().sum(dim=-2)
    return w1.mean(dim=-1)
