"""The kernels on layer lists other than the RAVE-like ones: the seeded
random graphs of the CPU planning tests (dilated, strided and transposed
convolutions with uneven pads and crops, residual units whose merges are
fused or not, three-branch heads with noise), streamed through the library
over a random partition into whole steps and compared element by element with
the oracle's causal model:
* FP32 at the drawn widths (2 to 4 channels: the narrow and GEMV FFMA kernels);
* BF16 at 64 channels (every convolution on tcgen05: strided layers gather
  their window rows, transposed ones run polyphase, merges unfused where a
  branch output has another reader);
* BF16 at 48 channels (no layer has whole 64-wide K slices: a BF16 model whose
  layers all take the FP32 kernels, which must then keep the FP32 bar)."""
import numpy as np
import pytest

from oracle import metrics
from oracle import model as M
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W
from test_random_graphs import random_graph

pytestmark = pytest.mark.gpu


def _stream(nodes, p, dtype, seed, cuda, n_steps=12):
    import torch

    info = M.analyze(nodes)
    step = info["in_per_step"]
    rng = np.random.default_rng(1000 + seed)
    x = rng.standard_normal((step * n_steps, nodes[0]["c_out"]))
    cuts, left = [], n_steps
    while left:
        n = int(rng.integers(1, min(left, 4) + 1))
        cuts.append(n)
        left -= n
    model = api.Model(nodes, p, dtype=dtype, max_streams=2, max_steps_per_call=4)
    s = model.stream(seed=seed)
    io = model.io
    outs, pos = [], 0
    for n in cuts:
        xb = torch.tensor(x[pos * step:(pos + n) * step], dtype=torch.float32, device=cuda)
        yb = torch.empty((n * io["out_per_step"], io["out_channels"]), dtype=torch.float32, device=cuda)
        s.process(xb, yb)
        outs.append(yb.cpu().numpy())
        pos += n
    assert model.device_status() == 0
    model.close()
    return np.concatenate(outs).astype(np.float64), M.run_causal(nodes, p, x, seed=seed)


@pytest.mark.parametrize("seed", list(range(10)))
def test_random_graph_fp32(cclib, cuda, seed):
    nodes = random_graph(seed)
    p = W.init_params(nodes, 100 + seed)
    out, ref = _stream(nodes, p, "f32", seed, cuda)
    err = metrics.max_abs(ref, out)
    assert err <= 1e-5 * metrics.rms(ref), f"seed {seed}: max-abs {err:.3e}, rms {metrics.rms(ref):.3e}"


@pytest.mark.parametrize("seed", list(range(10)))
def test_random_graph_bf16_tensor_cores(cclib, cuda, seed):
    nodes = random_graph(seed, channels=64)
    p = W.init_params(nodes, 100 + seed)
    out, ref = _stream(nodes, p, "bf16", seed, cuda)
    snr = metrics.snr_db(ref, out)
    err = metrics.max_abs(ref, out)
    assert snr >= 35.0 and err <= 2e-2 * np.max(np.abs(ref)), f"seed {seed}: SNR {snr:.1f} dB, max-abs {err:.3e}"


@pytest.mark.parametrize("seed", [10, 11, 12, 13])
def test_random_graph_bf16_model_on_fp32_kernels(cclib, cuda, seed):
    nodes = random_graph(seed, channels=48)
    p = W.init_params(nodes, 100 + seed)
    out, ref = _stream(nodes, p, "bf16", seed, cuda)
    err = metrics.max_abs(ref, out)
    assert err <= 1e-5 * metrics.rms(ref), f"seed {seed}: max-abs {err:.3e}, rms {metrics.rms(ref):.3e}"
