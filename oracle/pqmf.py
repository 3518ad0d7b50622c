"""Cosine-modulated pseudo-QMF bank (the RAVE-like model's multiband front/back end).

The paper names RAVE (section 2.3) but does not define its PQMF; this file is
the textbook construction (Nguyen 1994; Vaidyanathan, "Multirate Systems and
Filter Banks", 1993, ch. 8) with a Kaiser-window prototype whose cutoff is set
by the Lin & Vaidyanathan (1998) criterion.  Parity of this design is checked
by properties (near-perfect reconstruction, time-reversal and modulation
identities), not against the paper.

Definitions, for M bands and N taps, centre c = (N-1)/2:

    prototype  p[n] = kaiser_beta[n] * sin(wc (n - c)) / (pi (n - c))
    analysis   h_b[n] = 2 p[n] cos((2b+1) pi/(2M) (n - c) + (-1)^b pi/4)
    synthesis  g_b[n] = 2 p[n] cos((2b+1) pi/(2M) (n - c) - (-1)^b pi/4)

The cutoff wc minimises |r(2Ml)| / r(0), l != 0, where r is the prototype's
autocorrelation (the power-complementarity condition of a near-PR bank; for
N <= 4M the only such lag inside the support is 2M).

As layers of the model (cross-correlation, Eq. 1): the analysis is a strided
Conv(1 -> M, K=N, S=M, pad (N-M)/2 each side) whose kernel is g_b (correlating
with g_b convolves with its time reverse h_b), and the synthesis is a
ConvT(M -> 1, K=N, S=M, crop (N-M)/2) whose kernel is M * g_b.
"""
from __future__ import annotations

import numpy as np

DEFAULT_BETA = 5.0


def kaiser(n_taps, beta):
    """Kaiser window w[n] = I0(beta sqrt(1 - (2n/(N-1) - 1)^2)) / I0(beta), the
    PQMF prototype's window (Lin & Vaidyanathan 1998)."""
    n = np.arange(n_taps)
    arg = 1.0 - (2.0 * n / (n_taps - 1) - 1.0) ** 2
    return np.i0(beta * np.sqrt(np.maximum(arg, 0.0))) / np.i0(beta)


def prototype(n_taps, wc, beta):
    """Kaiser-windowed sinc prototype of cutoff wc (the PQMF of section 2.3's RAVE-like model)."""
    c = (n_taps - 1) / 2.0
    m = np.arange(n_taps) - c
    with np.errstate(invalid="ignore", divide="ignore"):
        ideal = np.where(m == 0, wc / np.pi, np.sin(wc * m) / (np.pi * m))
    return ideal * kaiser(n_taps, beta)


def _lag_error(n_taps, bands, wc, beta):
    p = prototype(n_taps, wc, beta)
    r = np.correlate(p, p, mode="full")  # lag l at index n_taps-1+l
    lags = [l for l in range(2 * bands, n_taps, 2 * bands)]
    r0 = r[n_taps - 1]
    return max(abs(r[n_taps - 1 + l]) for l in lags) / r0 if lags else 0.0


def design_cutoff(n_taps, bands, beta, grid=4000):
    """wc minimising the normalised autocorrelation at lags 2M*l (Lin &
    Vaidyanathan 1998), by a grid scan refined with golden-section search.  The
    search stays in [0.3 pi/M, pi/M], around the band edge pi/(2M): the
    criterion has further zeros at wider cutoffs that give no reconstruction."""
    lo, hi = 0.3 * np.pi / bands, 1.0 * np.pi / bands
    ws = np.linspace(lo, hi, grid)
    errs = [_lag_error(n_taps, bands, w, beta) for w in ws]
    i = int(np.argmin(errs))
    a, b = ws[max(i - 1, 0)], ws[min(i + 1, grid - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    for _ in range(200):
        c1, c2 = b - g * (b - a), a + g * (b - a)
        if _lag_error(n_taps, bands, c1, beta) < _lag_error(n_taps, bands, c2, beta):
            b = c2
        else:
            a = c1
    return 0.5 * (a + b)


def design(bands=16, n_taps=64, beta=DEFAULT_BETA):
    """The PQMF of section 2.3 (Nguyen 1994; Lin & Vaidyanathan 1998).  Returns
    (h, g, p, wc): analysis / synthesis filters [bands][n_taps], prototype."""
    wc = design_cutoff(n_taps, bands, beta)
    p = prototype(n_taps, wc, beta)
    c = (n_taps - 1) / 2.0
    n = np.arange(n_taps)
    h = np.empty((bands, n_taps))
    g = np.empty((bands, n_taps))
    for b in range(bands):
        theta = (2 * b + 1) * np.pi / (2 * bands) * (n - c)
        phase = (-1) ** b * np.pi / 4
        h[b] = 2 * p * np.cos(theta + phase)
        g[b] = 2 * p * np.cos(theta - phase)
    return h, g, p, wc


def analysis_weights(g):
    """Conv(1 -> M) kernel [M][1][N] of the analysis layer (section 2.3's multiband decomposition)."""
    return g[:, None, :].copy()


def synthesis_weights(g):
    """ConvT(M -> 1) kernel [M][1][N] of the synthesis layer (section 2.3's multiband recomposition)."""
    bands = g.shape[0]
    return (bands * g)[:, None, :].copy()
