"""Pins for the gradient reference (oracle/autodiff.py): its forward equals the
numpy causal model, and its gradients match central finite differences of the
numpy causal model."""
import numpy as np
import pytest
import torch

from oracle import autodiff as AD
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import workloads as W


def small_decoder(seed=0):
    nodes = W.rave_decoder(latent=8, capacity=4, ratios=(2, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    p = W.init_params(nodes, seed)
    _, g, _, _ = pqmf.design(4, 16, 5.0)
    p[W.pqmf_node_index(nodes)] = (pqmf.synthesis_weights(g), None)
    return nodes, p


def small_autoencoder(seed=0):
    enc = W.rave_encoder(latent=8, capacity=4, ratios=(2, 2), bands=4, pqmf_taps=16)
    dec = W.rave_decoder(latent=8, capacity=4, ratios=(2, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    nodes = W.chain(enc, dec)
    p = W.init_params(nodes, seed)
    _, g, _, _ = pqmf.design(4, 16, 5.0)
    for i, nd in enumerate(nodes):
        if nd["name"] == "pqmf":
            p[i] = (pqmf.analysis_weights(g), None)
        if nd["name"] == "ipqmf":
            p[i] = (pqmf.synthesis_weights(g), None)
    return nodes, p


@pytest.mark.parametrize("builder,frames,cin", [(W.tiny_stack, 40, 16), (small_decoder, 6, 8),
                                                (small_autoencoder, 64 * 3, 1)])
def test_torch_forward_equals_numpy_causal(builder, frames, cin):
    out = builder()
    nodes, p = out if isinstance(out, tuple) else (out, W.init_params(out, 0))
    x = W.signal(1, frames, cin)
    ref = M.run_causal(nodes, p, x, seed=3)
    pt = {i: (torch.tensor(w), None if b is None else torch.tensor(b)) for i, (w, b) in p.items()}
    y = AD.causal_forward(nodes, pt, torch.tensor(x.T.copy()), seed=3).detach().numpy().T
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def _fd(nodes, p, x, r, which, direction, h=1e-6):
    """Central finite difference of L = sum(r * y) along `direction`."""
    def loss(eps):
        xx, pp = x, dict(p)
        if which == "x":
            xx = x + eps * direction
        else:
            i, part = which
            w, b = p[i]
            pp[i] = (w + eps * direction, b) if part == 0 else (w, b + eps * direction)
        return float(np.sum(r * M.run_causal(nodes, pp, xx, seed=3)))
    return (loss(h) - loss(-h)) / (2 * h)


@pytest.mark.parametrize("builder,frames,cin", [(small_decoder, 5, 8), (small_autoencoder, 64 * 2, 1)])
def test_torch_gradients_match_finite_differences(builder, frames, cin):
    nodes, p = builder()
    x = W.signal(2, frames, cin)
    y = M.run_causal(nodes, p, x, seed=3)
    r = np.random.default_rng(5).standard_normal(y.shape)
    _, gx, gw = AD.gradients(nodes, p, x, r, seed=3)
    rng = np.random.default_rng(6)
    d = rng.standard_normal(x.shape)
    assert abs(_fd(nodes, p, x, r, "x", d) - np.sum(gx * d)) < 1e-6 * (1 + abs(np.sum(gx * d)))
    for i in sorted(p)[:: max(1, len(p) // 5)]:
        w, b = p[i]
        d = rng.standard_normal(w.shape)
        assert abs(_fd(nodes, p, x, r, (i, 0), d) - np.sum(gw[i][0] * d)) < 1e-6 * (1 + abs(np.sum(gw[i][0] * d)))
        if b is not None:
            d = rng.standard_normal(b.shape)
            assert abs(_fd(nodes, p, x, r, (i, 1), d) - np.sum(gw[i][1] * d)) < 1e-6 * (1 + abs(np.sum(gw[i][1] * d)))
