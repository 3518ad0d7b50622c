"""Pins for the oracle's cached-padding streaming (Fig. 1, section 2.2) and the
exactness claim of section 4.2: streamed == causal offline for every buffer
partition (E1), and causal offline == original delayed by the computed latency
on the interior (E2)."""
import numpy as np
import pytest

from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import workloads as W


def _decoder(seed=1):
    dec = W.rave_decoder()
    p = W.init_params(dec, seed)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    return dec, p


def _encoder(seed=4):
    enc = W.rave_encoder()
    p = W.init_params(enc, seed)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(enc)] = (pqmf.analysis_weights(g), None)
    return enc, p


@pytest.mark.parametrize("partition", [[512] * 8, [1] * 40 + [4056], [7, 100, 1, 3000, 988],
                                       W.buffer_partition(4096, 9, [1, 5, 64, 333])])
def test_tiny_stream_equals_causal_offline(partition):
    nodes = W.tiny_stack()
    p = W.init_params(nodes, 0)
    x = W.signal(0, 4096, 16)
    yc = M.run_causal(nodes, p, x)
    ys = M.Stream(nodes, p).run(x, partition)
    np.testing.assert_allclose(ys, yc, rtol=0, atol=1e-12 * np.abs(yc).max())


def test_tiny_causal_equals_original_delayed_on_interior():
    nodes = W.tiny_stack()
    p = W.init_params(nodes, 0)
    x = W.signal(0, 4096, 16)
    d = M.analyze(nodes)["delay"]
    w = M.warmup_frames(nodes)
    yc, yo = M.run_causal(nodes, p, x), M.run_original(nodes, p, x)
    np.testing.assert_array_equal(yc[d + w:], yo[w:len(yo) - d])
    # the warm-up region really differs (bias pre-roll replaces inner zero pads)
    assert not np.array_equal(yc[d:d + w], yo[:w])


def test_decoder_stream_equals_causal_offline():
    dec, p = _decoder()
    z = W.signal(1, 10, 128)
    yc = M.run_causal(dec, p, z, seed=77)
    for part in ([1] * 10, [3, 1, 6], [10]):
        ys = M.Stream(dec, p, seed=77).run(z, part)
        assert ys.shape == (10 * 2048, 1)
        np.testing.assert_allclose(ys, yc, rtol=0, atol=1e-12 * np.abs(yc).max())


def test_decoder_causal_equals_original_delayed():
    dec, p = _decoder()
    z = W.signal(2, 16, 128)
    yc = M.run_causal(dec, p, z, seed=3)
    yo = M.run_original(dec, p, z, seed=3)
    d = M.analyze(dec)["delay"]
    w = M.warmup_frames(dec)
    assert len(yo) - d - w > 4000
    np.testing.assert_allclose(yc[d + w:], yo[w:len(yo) - d], rtol=0, atol=1e-12)


def test_decoder_noise_off_reproduces_deterministic_heads():
    dec, p = _decoder()
    z = W.signal(2, 4, 128)
    a = M.run_causal(dec, p, z, seed=3, noise_on=False)
    b = M.run_causal(dec, p, z, seed=99, noise_on=False)
    np.testing.assert_array_equal(a, b)
    c = M.run_causal(dec, p, z, seed=99, noise_on=True)
    assert not np.array_equal(a, c)


def test_encoder_stream_equals_causal_and_original():
    enc, p = _encoder()
    x = W.signal(4, 2048 * 10, 1, std=0.1)
    yc = M.run_causal(enc, p, x)
    ys = M.Stream(enc, p).run(x, [2048, 4096, 2048 * 3, 2048 * 4])
    np.testing.assert_allclose(ys, yc, rtol=0, atol=1e-12 * np.abs(yc).max())
    yo = M.run_original(enc, p, x)
    d = M.analyze(enc)["delay"]
    w = M.warmup_frames(enc)
    assert len(yo) - d - w >= 2
    np.testing.assert_allclose(yc[d + w:], yo[w:len(yo) - d], rtol=0, atol=1e-12)


def test_stream_rejects_partial_step():
    enc, p = _encoder()
    with pytest.raises(ValueError):
        M.Stream(enc, p).process(np.zeros((1000, 1)))


def test_linear_shift_invariance_without_activations():
    """With identity activations and no biases the streamed model is linear and
    time-invariant: delaying the input by one step unit delays the output."""
    nodes = W.strip_activations(W.tiny_stack())
    p = {i: (w, np.zeros_like(b)) for i, (w, b) in W.init_params(nodes, 1).items()}
    x = W.signal(8, 600, 16)
    y = M.Stream(nodes, p).run(x, [100] * 6)
    xs = np.concatenate([np.zeros((13, 16)), x[:-13]])
    ys = M.Stream(nodes, p).run(xs, [37, 563])
    np.testing.assert_allclose(ys[13:], y[:-13], atol=1e-12)
    y2 = M.Stream(nodes, p).run(2.0 * x + xs, [600])
    np.testing.assert_allclose(y2, 2.0 * y + ys, atol=1e-11)


def test_chain_equals_encoder_then_decoder_without_noise():
    """The audio -> audio chain (one layer list) computes the encoder followed
    by the decoder on the same weights; with the noise branch off the two are
    the same arithmetic.  (With noise on they differ only by the noise
    index: the chain's heads see the encoder's delay in their aligned frame
    index.)"""
    enc = W.rave_encoder(latent=8, capacity=4, ratios=(2, 2), bands=4, pqmf_taps=16)
    dec = W.rave_decoder(latent=8, capacity=4, ratios=(2, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    nodes = W.chain(enc, dec)
    p = W.init_params(nodes, 5)
    off = len(enc) - 1
    pe = {i: p[i] for i in range(len(enc)) if i in p}
    pd = {k: p[off + k] for k in range(1, len(dec)) if off + k in p}
    x = W.signal(6, 64 * 5, 1, std=0.1)
    y_chain = M.run_causal(nodes, p, x, noise_on=False)
    y_two = M.run_causal(dec, pd, M.run_causal(enc, pe, x), noise_on=False)
    assert np.array_equal(y_chain, y_two)
    info_e, info_d, info_c = M.analyze(enc), M.analyze(dec), M.analyze(nodes)
    assert info_c["delay"] == info_e["delay"] * 16 + info_d["delay"]  # 16 samples per latent frame
