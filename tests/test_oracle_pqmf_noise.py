"""Pins for the PQMF design (properties) and the SplitMix64 noise (published vectors)."""
import os

import numpy as np
import pytest

from oracle import conv as C
from oracle import noise, pqmf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _reconstruction_snr(bands, taps, beta, seed=0):
    x = np.random.default_rng(seed).standard_normal(bands * 600)
    _, g, _, _ = pqmf.design(bands, taps, beta)
    half = (taps - bands) // 2
    sub = C.conv1d(x[None, :], pqmf.analysis_weights(g), None, bands, 1, half, half)
    y = C.conv_transpose_full(sub, pqmf.synthesis_weights(g), bands)[0, half:half + x.size]
    sl = slice(4 * taps, -4 * taps)
    return 10 * np.log10(np.sum(x[sl] ** 2) / np.sum((y - x)[sl] ** 2))


def test_pqmf_structure():
    h, g, p, wc = pqmf.design(16, 64)
    np.testing.assert_allclose(p, p[::-1], atol=1e-15)              # linear phase
    np.testing.assert_allclose(g, h[:, ::-1], atol=1e-14)           # g_b = time reverse of h_b
    # cosine modulation: h_b + g_b = 4 p cos(theta_b) cos(pi/4)
    n = np.arange(64) - 31.5
    for b in range(16):
        theta = (2 * b + 1) * np.pi / 32 * n
        np.testing.assert_allclose(h[b] + g[b], 4 * p * np.cos(theta) * np.cos(np.pi / 4), atol=1e-14)
    assert 0.3 * np.pi / 16 < wc < np.pi / 16
    r = np.correlate(p, p, "full")
    assert abs(r[63 + 32]) < 1e-6 * r[63]                            # Lin-Vaidyanathan criterion


def test_pqmf_near_perfect_reconstruction_longer_prototype():
    """The same construction reconstructs to > 50 dB with 128 taps."""
    assert _reconstruction_snr(16, 128, 8.0) > 50.0


def test_pqmf_reconstruction_at_configured_size():
    """16 bands x 64 taps (4 taps per band and phase): measured ~22.8 dB, a
    property of such a short prototype."""
    snr = _reconstruction_snr(16, 64, pqmf.DEFAULT_BETA)
    assert 21.0 < snr < 30.0


def _golden():
    seeds, vals, buckets = None, [], None
    with open(os.path.join(GOLDEN, "splitmix64_rosetta.txt")) as f:
        lines = [l.strip() for l in f if l.strip() and not l.startswith("#")]
    seed = int(lines[0].split()[1])
    vals = [int(v) for v in lines[1:6]]
    _, bseed, bcount, bk = lines[6].split()
    counts = [int(v) for v in lines[7].split()]
    return seed, vals, int(bseed), int(bcount), int(bk), counts


def test_splitmix64_published_vectors():
    seed, vals, bseed, bcount, bk, counts = _golden()
    assert noise.splitmix64_sequence(seed, 5) == vals
    # counter form: draw(seed, n) is the (n+1)-th output
    assert [noise.draw(seed, i) for i in range(5)] == vals
    got = [0] * bk
    for z in noise.splitmix64_sequence(bseed, bcount):
        got[(z * bk) >> 64] += 1
    assert got == counts


def test_noise_uniform_range_and_float32_exact():
    u = noise.uniform_block(123, -50, 200, 16)
    assert u.min() >= -1.0 and u.max() < 1.0
    np.testing.assert_array_equal(u.astype(np.float32).astype(np.float64), u)
    assert abs(u.mean()) < 0.05
    # keyed on (band, frame) only: a window starting elsewhere sees the same values
    np.testing.assert_array_equal(noise.uniform_block(123, 0, 10, 16), u[50:60])
