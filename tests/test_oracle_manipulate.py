"""Pins for the oracle's latent manipulation (sections 5.1 and 5.2):

* the identity and Fig. 7's two controls (bias one dimension, replace another)
  are exact;
* the noise term is the sequential SplitMix64 generator (itself pinned to the
  published vectors) read in counter order t * channels + c from the tagged
  seed, so a transposed counter, a dropped tag or a wrong offset fails;
* it is buffer-partition invariant (the property streaming relies on) and
  has the uniform law on [-1, 1);
* streamed through the oracle's cached-padding stream with controls that
  change between buffers, the output equals the causal offline model on the
  manipulated input."""
import numpy as np

from oracle import manipulate as MP
from oracle import model as M
from oracle import noise
from paper_2204_07064_gb300 import workloads as W


def test_identity_is_exact():
    x = W.signal(0, 40, 12)
    assert np.array_equal(MP.manipulate(x), x)
    assert np.array_equal(MP.manipulate(x, np.ones(12), np.zeros(12), np.zeros(12), seed=9), x)


def test_fig7_bias_first_and_replace_last_dimension():
    x = W.signal(1, 30, 8)
    scale = np.ones(8)
    bias = np.zeros(8)
    bias[0] = 1.75
    scale[-1], bias[-1] = 0.0, -0.4
    y = MP.manipulate(x, scale, bias)
    assert np.array_equal(y[:, 0], x[:, 0] + 1.75)
    assert np.array_equal(y[:, -1], np.full(30, -0.4))
    assert np.array_equal(y[:, 1:-1], x[:, 1:-1])


def test_noise_is_the_tagged_splitmix64_sequence_in_counter_order():
    seed, T, C = 0x1234_5678_9ABC_DEF0, 7, 5
    seq = noise.splitmix64_sequence(seed ^ MP.TAG, T * C)
    want = np.array([(z >> 40) * 2.0 ** -23 - 1.0 for z in seq]).reshape(T, C)
    assert np.array_equal(MP.input_noise(seed, 0, T, C), want)
    # an offset t0 continues the same sequence
    assert np.array_equal(MP.input_noise(seed, 3, 4, C), want[3:])
    # the heads' generator of the same seed (no tag) draws other values
    heads = noise.uniform_block(seed, 0, T, C)
    assert not np.any(heads == want)


def test_noise_amplitude_and_partition_invariance():
    seed, T, C = 77, 64, 16
    x = W.signal(2, T, C)
    amp = np.linspace(0.0, 0.5, C)
    whole = MP.manipulate(x, 0.5, 0.1, amp, seed=seed)
    parts = [MP.manipulate(x[a:b], 0.5, 0.1, amp, seed=seed, t0=a) for a, b in ((0, 5), (5, 32), (32, 64))]
    assert np.array_equal(np.concatenate(parts), whole)
    u = MP.input_noise(seed, 0, T, C)
    np.testing.assert_allclose(whole, 0.5 * x + 0.1 + amp * u, rtol=0, atol=1e-15)
    assert np.all(whole[:, 0] == 0.5 * x[:, 0] + 0.1)  # zero amplitude adds nothing


def test_noise_law_uniform():
    u = MP.input_noise(5, 0, 2000, 16)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01
    assert abs(u.var() - 1.0 / 3.0) < 0.01
    c = np.corrcoef(u.T)
    assert np.max(np.abs(c - np.eye(16))) < 0.08  # channels are not correlated


def test_piecewise_controls():
    p = MP.piecewise(6, 2, [(2, [1.0, 2.0]), (4, 3.0)], default=0.0)
    assert p.tolist() == [[0, 0], [0, 0], [1, 2], [1, 2], [3, 3], [3, 3]]


def test_streamed_with_changing_controls_equals_offline_on_manipulated_input():
    nodes = W.rave_decoder(latent=8, capacity=4, ratios=(2, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    p = W.init_params(nodes, 3)
    T, C, seed = 12, 8, 21
    z = W.signal(4, T, C)
    bias = MP.piecewise(T, C, [(4, np.r_[1.5, np.zeros(7)])], 0.0)
    scale = MP.piecewise(T, C, [(8, np.r_[np.ones(7), 0.0])], 1.0)
    amp = MP.piecewise(T, C, [(6, 0.3)], 0.0)
    zm = MP.manipulate(z, scale, bias, amp, seed=seed)
    s = M.Stream(nodes, p, seed=seed)
    out, pos = [], 0
    for n in (3, 1, 4, 4):  # controls change inside and at buffer edges
        out.append(s.process(MP.manipulate(z[pos:pos + n], scale[pos:pos + n], bias[pos:pos + n],
                                           amp[pos:pos + n], seed=seed, t0=pos)))
        pos += n
    np.testing.assert_allclose(np.concatenate(out), M.run_causal(nodes, p, zm, seed=seed), rtol=0, atol=1e-12)
