"""Distances of section 4.2 and the acceptance checks used by the parity tests.

* Eq. 5, waveform distance  L_w(x, y) = ||x - y||_2
* Eq. 4, spectral distance  L_s(x, y) = ||log(S(x) + eps) - log(S(y) + eps)||_2,
  S the amplitude STFT, eps = 1 (section 4.2).  The STFT parameters are not
  given in the paper; this file reads them as a 2048-point Hann window with
  hop 512 (no padding).
* SNR in dB, max-abs error relative to the reference peak or RMS.
"""
from __future__ import annotations

import numpy as np


def waveform_distance(x, y):
    """Eq. 5: waveform distance L_w(x, y) = ||x - y||_2 (section 4.2)."""
    return float(np.sqrt(np.sum((np.asarray(x, np.float64) - np.asarray(y, np.float64)) ** 2)))


def amplitude_stft(x, n_fft=2048, hop=512):
    """Amplitude STFT S of Eq. 4 (section 4.2), read as a 2048-point periodic
    Hann window with hop 512."""
    x = np.asarray(x, np.float64).ravel()
    n = np.arange(n_fft)
    win = np.sin(np.pi * n / n_fft) ** 2  # periodic Hann, the window of section 3.3
    frames = 1 + max(0, (x.size - n_fft) // hop)
    spec = np.empty((frames, n_fft // 2 + 1))
    for f in range(frames):
        seg = x[f * hop:f * hop + n_fft]
        if seg.size < n_fft:
            seg = np.pad(seg, (0, n_fft - seg.size))
        spec[f] = np.abs(np.fft.rfft(seg * win))
    return spec


def spectral_distance(x, y, eps=1.0, n_fft=2048, hop=512):
    """Eq. 4: spectral distance ||log(S(x) + eps) - log(S(y) + eps)||_2,
    eps = 1 (section 4.2)."""
    sx = amplitude_stft(x, n_fft, hop)
    sy = amplitude_stft(y, n_fft, hop)
    return float(np.sqrt(np.sum((np.log(sx + eps) - np.log(sy + eps)) ** 2)))


def snr_db(ref, out):
    """SNR of `out` against `ref` in dB: the low-precision parity bar (no
    paper passage; the paper's forms are FP32)."""
    ref = np.asarray(ref, np.float64)
    err = np.asarray(out, np.float64) - ref
    den = np.sum(err ** 2)
    return float("inf") if den == 0 else float(10.0 * np.log10(np.sum(ref ** 2) / den))


def rms(x):
    """Root mean square, the scale of the FP32 parity bar (no paper passage)."""
    x = np.asarray(x, np.float64)
    return float(np.sqrt(np.mean(x ** 2)))


def max_abs(ref, out):
    """Largest absolute difference, the element-wise parity check (no paper passage)."""
    return float(np.max(np.abs(np.asarray(out, np.float64) - np.asarray(ref, np.float64))))
