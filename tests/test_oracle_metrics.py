"""Pins of the oracle's Eq. 4 / Eq. 5 distances (section 4.2) and of the
start-up boundary ``warmup_frames`` from both sides.

Closed forms used:
* a periodic Hann window of N points has sum N/2, and its DFT has exactly three
  non-zero bins (0, +-1) of weights 1/2, -1/4, -1/4; so a cosine of amplitude A
  centred on bin k0 has |S| = A*N/4 at k0, A*N/8 at k0 +- 1 and 0 elsewhere
  (a rectangular window would give A*N/2 and zeros);
* a unit impulse at sample m lands in every frame f with f*hop <= m < f*hop + N
  with the flat magnitude win[m - f*hop] in every bin (pins hop and alignment);
* L_s(x, x) = 0 and, since S(0) = 0 and log(0 + 1) = 0, L_s(x, 0) = ||log(S(x) + 1)||;
* L_w(x, 2x) = ||x||.
"""
import numpy as np
import pytest

from oracle import metrics as Q
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import workloads as W


def _cosine(A, k0, n_fft, length):
    n = np.arange(length)
    return A * np.cos(2 * np.pi * k0 * n / n_fft)


def test_stft_bin_centred_cosine_closed_form():
    n_fft, A, k0 = 2048, 0.7, 100
    S = Q.amplitude_stft(_cosine(A, k0, n_fft, n_fft))
    assert S.shape == (1, n_fft // 2 + 1)
    want = np.zeros(n_fft // 2 + 1)
    want[k0], want[k0 - 1], want[k0 + 1] = A * n_fft / 4, A * n_fft / 8, A * n_fft / 8
    np.testing.assert_allclose(S[0], want, rtol=0, atol=1e-9 * A * n_fft)


def test_stft_impulse_pins_hop_and_window_alignment():
    n_fft, hop = 2048, 512
    x = np.zeros(n_fft + 3 * hop)
    m = 1500
    x[m] = 1.0
    S = Q.amplitude_stft(x)
    assert S.shape[0] == 4  # 1 + (len - N) // hop frames, no padding
    n = np.arange(n_fft)
    win = np.sin(np.pi * n / n_fft) ** 2
    for f in range(4):
        inside = f * hop <= m < f * hop + n_fft
        want = win[m - f * hop] if inside else 0.0
        np.testing.assert_allclose(S[f], np.full(n_fft // 2 + 1, want), rtol=0, atol=1e-12)


def test_spectral_distance_closed_forms():
    n_fft, A, k0 = 2048, 0.3, 37
    x = _cosine(A, k0, n_fft, n_fft)
    assert Q.spectral_distance(x, x) == 0.0
    # S(0) = 0 and eps = 1: only the three bins of the cosine contribute
    want = np.sqrt(np.log(A * n_fft / 4 + 1) ** 2 + 2 * np.log(A * n_fft / 8 + 1) ** 2)
    assert Q.spectral_distance(x, np.zeros_like(x)) == pytest.approx(want, rel=1e-9)
    # log(S + eps), not log(S) + eps: doubling the amplitude changes each bin by
    # log((2a + 1) / (a + 1)), not by log 2
    want2 = np.sqrt(np.log((2 * A * n_fft / 4 + 1) / (A * n_fft / 4 + 1)) ** 2
                    + 2 * np.log((2 * A * n_fft / 8 + 1) / (A * n_fft / 8 + 1)) ** 2)
    assert Q.spectral_distance(x, 2 * x) == pytest.approx(want2, rel=1e-9)


def test_waveform_distance_closed_form():
    x = W.signal(3, 1000, 1).ravel()
    assert Q.waveform_distance(x, x) == 0.0
    assert Q.waveform_distance(x, 2 * x) == pytest.approx(np.sqrt(np.sum(x ** 2)), rel=1e-12)


def _first_exact(yc, yo, d, atol):
    """Count of leading frames t where causal[t + d] != original[t]."""
    n = len(yo) - d
    diff = np.abs(yc[d:d + n] - yo[:n]).max(axis=1)
    bad = np.nonzero(diff > atol)[0]
    return int(bad.max() + 1) if len(bad) else 0, diff


def _decoder():
    dec = W.rave_decoder()
    p = W.init_params(dec, 1)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    return dec, p


@pytest.mark.parametrize("case", ["tiny", "decoder", "encoder"])
def test_warmup_frames_is_tight(case):
    """E2's interior starts exactly at warmup_frames: the frame there and every
    later one equal the delayed original bit for bit, and the frame just before
    differs (random weights have no zero tap), so the bound is neither too
    small nor too large."""
    if case == "tiny":
        nodes = W.tiny_stack()
        p = W.init_params(nodes, 0)
        x = W.signal(0, 512, 16)
        seed, atol = 0, 0.0
    elif case == "decoder":
        nodes, p = _decoder()
        x = W.signal(2, 12, 128)
        seed, atol = 3, 0.0
    else:
        nodes = W.rave_encoder()
        p = W.init_params(nodes, 5)
        _, g, _, _ = pqmf.design(16, 64)
        p[W.pqmf_node_index(nodes)] = (pqmf.analysis_weights(g), None)
        x = W.signal(4, 2048 * 12, 1, std=0.1)
        seed, atol = 0, 0.0
    yc = M.run_causal(nodes, p, x, seed=seed)
    yo = M.run_original(nodes, p, x, seed=seed)
    d = M.analyze(nodes)["delay"]
    w = M.warmup_frames(nodes)
    assert w > 0
    got, diff = _first_exact(yc, yo, d, atol)
    assert got == w
    # the same arithmetic from frame w on: bit-identical, while frame w - 1
    # still carries the causal pre-roll (far from the start only faintly)
    assert diff[w - 1] > 0.0
    assert np.all(diff[w:] == 0.0)
