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


def wide_strided_stack(seed=0):
    """Layers wide enough for the tiled backward kernels, with the strides of
    the encoder and decoder: a stride-4 conv (K=8) and a stride-2 conv (K=5,
    so residues meet different tap counts), a stride-4 transposed conv, a
    dilated conv (dilation 5) and a residual add."""
    n = W._node
    nodes = [W.input_node(32),
             n("conv", [0], 32, 64, k=8, stride=4, pad_left=2, pad_right=2, act_in=None, name="down4"),
             n("conv", [1], 64, 96, k=5, stride=2, pad_left=2, pad_right=2, act_in="leaky", name="down2"),
             n("convt", [2], 96, 64, k=8, stride=4, crop=2, act_in="leaky", name="up4"),
             n("conv", [3], 64, 64, k=3, dilation=5, pad_left=5, pad_right=5, act_in="leaky", name="dil"),
             n("add", [3, 4], 64, 64, bias=False, name="add"),
             n("conv", [5], 64, 48, k=3, pad_left=1, pad_right=1, act_in="leaky", name="out")]
    return nodes, W.init_params(nodes, seed)


@pytest.mark.parametrize("chunk", [1, 3])
def test_backward_wide_strided_layers(cclib, cuda, chunk):
    """FP32 parity of the tiled dW / dX kernels (split reductions, residue-
    ordered rows of strided convolutions, phases of a transposed one, a
    dilation above a chunk's output frames at 1-step chunks) against the
    oracle's gradient, the cache adjoint carried from chunk to chunk."""
    import torch

    nodes, p = wide_strided_stack(3)
    info = M.analyze(nodes)
    xs = [W.signal(50 + k, 12 * info["in_per_step"], 32) for k in range(3)]
    seeds = [1, 2, 3]
    y, gx, grads, r, _, _ = _run(nodes, p, xs, seeds, chunk, torch, cuda)
    gw_ref = {}
    for k in range(3):
        _, gxr, gwr = AD.gradients(nodes, p, xs[k], r[k], seed=seeds[k])
        _close(gx[k], gxr, f"dL/dx stream {k}")
        for i, (dw, db) in gwr.items():
            a = gw_ref.get(i)
            gw_ref[i] = (dw, db) if a is None else (a[0] + dw, None if db is None else a[1] + db)
    for i, (dw, db) in grads.items():
        _close(dw, gw_ref[i][0], f"dL/dw {nodes[i]['name']}")
        if db is not None:
            _close(db, gw_ref[i][1], f"dL/db {nodes[i]['name']}")


def test_weight_gradients_without_input_gradient(cclib, cuda):
    """An input that does not require a gradient: the backward still runs
    (the runner's weights anchor), skips the model input's adjoint (grad_x
    NULL), and every weight and bias gradient is the same, bit for bit."""
    import torch

    nodes, p = small_autoencoder()
    xs = [W.signal(40 + k, 96, 1) for k in range(2)]
    _, _, g_all, r, _, _ = _run(nodes, p, xs, [3, 4], 2, torch, cuda)
    model = api.Model(nodes, p, dtype="f32", max_streams=2, max_steps_per_call=2)
    runner = AG.StreamedRunner(model, p, [model.stream(seed=s) for s in (3, 4)], 2)
    x = torch.tensor(np.stack(xs), dtype=torch.float32, device=cuda)
    y = AG.streamed(x, runner)
    assert y.requires_grad and not x.requires_grad
    y.backward(torch.tensor(r, dtype=torch.float32, device=cuda))
    torch.cuda.synchronize()
    assert x.grad is None
    for i in p:
        dw, db = runner.grads.read(i)
        np.testing.assert_array_equal(dw, g_all[i][0])
        if db is not None:
            np.testing.assert_array_equal(db, g_all[i][1])


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


def bf16_decoder(seed=0):
    """A decoder wide enough for the tensor cores (256 -> 128 -> 64 channels),
    with the FP32 tail (narrow heads and inverse PQMF)."""
    nodes = W.rave_decoder(latent=16, capacity=64, ratios=(2, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    p = W.init_params(nodes, seed)
    _, g, _, _ = pqmf.design(4, 16, 5.0)
    p[W.pqmf_node_index(nodes)] = (pqmf.synthesis_weights(g), None)
    return nodes, p


def _tc_layers(nodes, fmt):
    """The layers the BF16/FP16 modes run on the tensor cores (the rule the
    library documents: a conv or convT with c_in % 64 == 0 and c_out % 8 == 0)."""
    return {i: fmt for i, nd in enumerate(nodes)
            if nd["op"] in ("conv", "convt") and nd["c_in"] % 64 == 0 and nd["c_out"] % 8 == 0}


def shallow_tc_stack(seed):
    """Every tensor-core layer kind in a few layers: LeakyReLU -> convT (K=4,
    S=2), a dilated k=3 conv and a 1x1 conv (both on LeakyReLU views), a
    residual add, and a k=3 conv on the add's plain low-precision view."""
    n = W._node
    nodes = [W.input_node(64),
             n("convt", [0], 64, 64, k=4, stride=2, crop=1, act_in="leaky", name="up"),
             n("conv", [1], 64, 64, k=3, dilation=3, pad_left=3, pad_right=3, act_in="leaky", name="a"),
             n("conv", [2], 64, 64, k=1, act_in="leaky", name="b"),
             n("add", [1, 3], 64, 64, bias=False, name="add"),
             n("conv", [4], 64, 64, k=3, pad_left=1, pad_right=1, act_in=None, name="c")]
    return nodes, W.init_params(nodes, seed)


def _streamed_gradients(cuda, nodes, p, dtype, xs, seeds, chunk, r_seed=12):
    import torch

    model = api.Model(nodes, p, dtype=dtype, max_streams=len(xs), max_steps_per_call=chunk, fuse_units=False)
    runner = AG.StreamedRunner(model, p, [model.stream(seed=s) for s in seeds], chunk)
    x = torch.tensor(np.stack(xs), dtype=torch.float32, device=cuda, requires_grad=True)
    y = AG.streamed(x, runner)
    r = np.random.default_rng(r_seed).standard_normal(tuple(y.shape))
    y.backward(torch.tensor(r, dtype=torch.float32, device=cuda))
    torch.cuda.synchronize()
    assert model.device_status() == 0
    grads = {i: runner.grads.read(i) for i in p}
    return x.grad.cpu().numpy(), grads, r


def _oracle_sums(nodes, p, xs, seeds, r, rounded):
    gx, gw = [], {}
    for k in range(len(xs)):
        _, gxr, gwr = AD.gradients(nodes, p, xs[k], r[k], seed=seeds[k], rounded=rounded)
        gx.append(gxr)
        for i, (dw, db) in gwr.items():
            a = gw.get(i)
            gw[i] = (dw, db) if a is None else (a[0] + dw, None if db is None else a[1] + db)
    return gx, gw


def _snr(g, ref):
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return 10 * np.log10(np.sum(ref ** 2) / max(np.sum((g - ref) ** 2), 1e-300))


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("pseed", [2, 3, 4])
def test_lowp_gradient_is_the_rounded_models(cclib, cuda, dtype, pseed):
    """Differentiation with a BF16 (FP16) forward on the tensor cores: the
    backward multiplies the rounded weights and activations the forward
    multiplied, so dL/dx and every dL/dw, dL/db equal the oracle's FP64
    gradients of the model with those operands rounded (activated inputs to
    nearest, weights row by row after scaling to max |w| = 1), over chunks
    whose cache adjoints carry from chunk to chunk: >= 70 dB and max-abs <=
    1e-3 x peak per tensor.  The model is shallow on purpose: the GPU sums in
    FP32 and the oracle in FP64, and once a value lands on the other side of a
    rounding boundary the two forwards part and the gap grows layer by layer
    (faster in FP16, whose grid is 8x finer), so only a few layers compare
    exactly; the deep decoder is checked below for what rounding costs."""
    nodes, p = shallow_tc_stack(pseed)
    frames, chunk = 6, 2
    xs = [W.signal(60 + k, frames, 64) for k in range(2)]
    seeds = [7, 8]
    gx, grads, r = _streamed_gradients(cuda, nodes, p, dtype, xs, seeds, chunk)
    gxr, gwr = _oracle_sums(nodes, p, xs, seeds, r, _tc_layers(nodes, dtype))

    def close(g, ref, what):
        snr = _snr(g, ref)
        rel = np.abs(np.asarray(g, np.float64) - ref).max() / max(np.abs(ref).max(), 1e-30)
        assert snr >= 70.0 and rel <= 1e-3, f"{dtype} {what}: SNR {snr:.1f} dB, max-abs/peak {rel:.2e}"

    for k in range(2):
        close(gx[k], gxr[k], f"dL/dx stream {k}")
    for i, (dw, db) in grads.items():
        close(dw, gwr[i][0], f"dL/dw {nodes[i]['name']}")
        if db is not None:
            close(db, gwr[i][1], f"dL/db {nodes[i]['name']}")


@pytest.mark.parametrize("dtype,min_cos", [("bf16", 0.98), ("f16", 0.995)])
def test_lowp_decoder_gradient_direction(cclib, cuda, dtype, min_cos):
    """What rounding costs a decoder's gradient: against the FP64 gradient of
    the exact model, every gradient tensor of the BF16 (FP16) decoder points
    the same way (cosine >= 0.98 / 0.995).  The error is mostly LeakyReLU
    derivatives taken on the other side of zero where rounding moved a value
    across it (a 0.2 vs 1 slope at that element), summed over the layers."""
    nodes, p = bf16_decoder(2)
    frames, chunk = 6, 2
    xs = [W.signal(60 + k, frames, 16) for k in range(2)]
    seeds = [7, 8]
    gx, grads, r = _streamed_gradients(cuda, nodes, p, dtype, xs, seeds, chunk)
    gxr, gwr = _oracle_sums(nodes, p, xs, seeds, r, None)

    def cos(g, ref, what):
        g = np.asarray(g, np.float64).ravel()
        ref = np.asarray(ref, np.float64).ravel()
        c = float(g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref)))
        assert c >= min_cos, f"{dtype} {what}: cosine {c:.4f}"

    for k in range(2):
        cos(gx[k], gxr[k], f"dL/dz stream {k}")
    for i, (dw, db) in grads.items():
        cos(dw, gwr[i][0], f"dL/dw {nodes[i]['name']}")
        if db is not None:
            cos(db, gwr[i][1], f"dL/db {nodes[i]['name']}")


def test_lowp_gradients_need_unfused_units(cclib, cuda):
    nodes, p = bf16_decoder(2)
    model = api.Model(nodes, p, dtype="bf16", max_streams=1, max_steps_per_call=1)
    with pytest.raises(api.CCError) as e:
        api.Grads(model, p)
    assert e.value.status == -7


def test_compact_checkpoint_restores_the_stream(cclib, cuda):
    """A checkpoint holds the step counter, the seed and the cached rows only
    (about a tenth of the arena slot for the decoder); restoring it into a
    stream that ran further makes that stream continue exactly as the
    original, in BF16 (mirrored low-precision rows included) and FP32."""
    import torch

    dec = W.rave_decoder()
    p = W.init_params(dec, 1)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    for dtype in ("bf16", "f32"):
        model = api.Model(dec, p, dtype=dtype, max_streams=3, max_steps_per_call=1)
        a, b, c = model.stream(seed=1), model.stream(seed=1), model.stream(seed=2)
        nb = api.snapshot_bytes(model)
        assert nb < model.state_bytes[1] / 4
        z = torch.tensor(W.signal(3, 40, 128)[:, None, :], dtype=torch.float32, device=cuda)
        y = torch.empty((1, 2048, 1), device=cuda)
        for t in range(13):
            model.process_batch([a, b], torch.stack([z[t], z[t]]), torch.empty((2, 2048, 1), device=cuda))
        buf = torch.empty(2 * nb, dtype=torch.uint8, device=cuda)
        api.snapshot_batch(model, [a, b], buf)
        for t in range(13, 31):  # b runs on: every ring wraps past the checkpoint's rows
            model.process_batch([b], z[t:t + 1], y)
        api.restore_batch(model, [c, b], buf)  # c takes a's state, b returns to it
        ya = torch.empty((1, 2048, 1), device=cuda)
        yb = torch.empty_like(ya)
        yc = torch.empty_like(ya)
        for t in range(13, 20):
            model.process_batch([a], z[t:t + 1], ya)
            model.process_batch([b], z[t:t + 1], yb)
            model.process_batch([c], z[t:t + 1], yc)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(yb.cpu().numpy(), ya.cpu().numpy())
            np.testing.assert_array_equal(yc.cpu().numpy(), ya.cpu().numpy())
        model.close()
