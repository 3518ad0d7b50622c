"""Differentiation form: the library's hand-written chunked backward (behind a
torch.autograd.Function) against the gradient of the causal model computed
by the oracle (torch float64 autograd, itself pinned to finite differences).

Loss L = sum(r * y) with a seeded r (a linear functional: its gradient is one
vector-Jacobian product).  Bar: max |g - g_ref| <= 1e-4 x max |g_ref| per tensor
(FP32 arithmetic against FP64)."""
import numpy as np
import pytest

from oracle import autodiff as AD
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import autograd as AG
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4


def _close(g, ref, what):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(g - ref).max()
    assert err <= GRAD_TOL * scale, f"{what}: max-abs {err:.3e} > {GRAD_TOL} x {scale:.3e}"


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


def _run(nodes, p, xs, seeds, chunk_steps, torch, dev):
    count = len(xs)
    model = api.Model(nodes, p, dtype="f32", max_streams=count, max_steps_per_call=chunk_steps)
    streams = [model.stream(seed=s) for s in seeds]
    runner = AG.StreamedRunner(model, p, streams, chunk_steps)
    x = torch.tensor(np.stack(xs), dtype=torch.float32, device=dev, requires_grad=True)
    y = AG.streamed(x, runner)
    r = np.random.default_rng(11).standard_normal(tuple(y.shape))
    y.backward(torch.tensor(r, dtype=torch.float32, device=dev))
    torch.cuda.synchronize()
    grads = {i: runner.grads.read(i) for i in p}
    return y.detach().cpu().numpy(), x.grad.cpu().numpy(), grads, r, model, runner


@pytest.mark.parametrize("builder,frames,chunk", [(small_decoder, 6, 2), (small_autoencoder, 96, 2)])
def test_backward_matches_oracle_gradient(cclib, cuda, builder, frames, chunk):
    import torch

    nodes, p = builder()
    cin = nodes[0]["c_in"]
    seeds = [3, 4]
    xs = [W.signal(20 + k, frames, cin) for k in range(2)]
    y, gx, grads, r, model, runner = _run(nodes, p, xs, seeds, chunk, torch, cuda)
    gw_ref = {i: (np.zeros_like(w), None if b is None else np.zeros_like(b)) for i, (w, b) in p.items()}
    for k in range(2):
        yref = M.run_causal(nodes, p, xs[k], seed=seeds[k])
        np.testing.assert_allclose(y[k], yref, rtol=0, atol=1e-5 * np.sqrt(np.mean(yref ** 2)))
        _, gxr, gwr = AD.gradients(nodes, p, xs[k], r[k], seed=seeds[k])
        _close(gx[k], gxr, f"dL/dx stream {k}")
        for i in gwr:
            gw_ref[i] = (gw_ref[i][0] + gwr[i][0], None if gwr[i][1] is None else gw_ref[i][1] + gwr[i][1])
    for i in p:
        _close(grads[i][0], gw_ref[i][0], f"dL/dw node {i} {nodes[i]['name']}")
        if gw_ref[i][1] is not None:
            _close(grads[i][1], gw_ref[i][1], f"dL/db node {i} {nodes[i]['name']}")


def test_gradient_independent_of_chunking(cclib, cuda):
    import torch

    nodes, p = small_decoder(1)
    xs = [W.signal(30, 6, 8)]
    _, g1, w1, _, _, _ = _run(nodes, p, xs, [5], 1, torch, cuda)
    _, g3, w3, _, _, _ = _run(nodes, p, xs, [5], 3, torch, cuda)
    _close(g3, g1, "dL/dx, chunks of 3 vs 1")
    for i in p:
        _close(w3[i][0], w1[i][0], f"dL/dw node {i}")


def test_full_decoder_latent_gradient(cclib, cuda):
    """The RAVE-like decoder (full widths), latent inversion: dL/dz and the
    gradients of a few layers against the oracle."""
    import torch

    dec = W.rave_decoder()
    p = W.init_params(dec, 2)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    z = [W.signal(40, 4, 128)]
    _, gz, grads, r, _, _ = _run(dec, p, z, [9], 1, torch, cuda)
    _, gzr, gwr = AD.gradients(dec, p, z[0], r[0], seed=9)
    _close(gz[0], gzr, "dL/dz")
    for i in (1, 2, 20, len(dec) - 1):
        if i in p:
            _close(grads[i][0], gwr[i][0], f"dL/dw node {i} {dec[i]['name']}")


def test_backward_restores_forward_state(cclib, cuda):
    """After forward + backward the streams continue exactly as after the
    forward alone."""
    import torch

    nodes, p = small_decoder(3)
    x = W.signal(50, 4, 8)
    model = api.Model(nodes, p, dtype="f32", max_streams=2, max_steps_per_call=2)
    a, b = model.stream(seed=1), model.stream(seed=1)
    runner = AG.StreamedRunner(model, p, [a], 2)
    xt = torch.tensor(x[None], dtype=torch.float32, device=cuda, requires_grad=True)
    AG.streamed(xt, runner).sum().backward()
    yb = torch.empty((1, 4 * model.io["out_per_step"], 1), device=cuda)
    model.process_batch([b], torch.tensor(x[None], dtype=torch.float32, device=cuda), yb)
    nxt = torch.tensor(W.signal(51, 2, 8)[None], dtype=torch.float32, device=cuda)
    ya = torch.empty((1, 2 * model.io["out_per_step"], 1), device=cuda)
    yb2 = torch.empty_like(ya)
    model.process_batch([a], nxt, ya)
    model.process_batch([b], nxt, yb2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ya.cpu().numpy(), yb2.cpu().numpy())
