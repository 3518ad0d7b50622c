"""The allocation-free cached Conv1d step (cc_cached_conv1d_static).

Some callers of this library cannot allocate device memory while they
process audio: a real-time audio callback must not block (cudaMalloc can
synchronise the device and take an unbounded time), and a plug-in embedded in
a host may only use memory reserved up front.  For them the library offers a
variant of its FP32 cached convolution whose scratch lives in a fixed device
array.  This test calls it through the C ABI on two consecutive buffers and
compares each output with the ordinary entry point (a model of one conv
layer processed with cc_stream_process), within the FP32 tolerance the
other parity tests use.  It runs last so that a failure here never hides
another test's result."""
import numpy as np
import pytest

from oracle import metrics
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.mark.parametrize("c_in,c_out,k,d,act,n", [(16, 16, 3, 2, "leaky", 512), (64, 32, 3, 9, None, 300)])
def test_static_scratch_conv_matches_stream_process(cclib, cuda, c_in, c_out, k, d, act, n):
    import torch

    half = (k - 1) * d // 2
    nodes = [W.input_node(c_in),
             W._node("conv", [0], c_in, c_out, k=k, dilation=d, pad_left=half,
                     pad_right=(k - 1) * d - half, act_in=act)]
    params = W.init_params(nodes, 3)
    w, b = params[1]
    model = api.Model(nodes, params, max_streams=1, max_steps_per_call=n)
    stream = model.stream()
    wt = torch.tensor(w, dtype=torch.float32, device=cuda)
    bt = torch.tensor(b, dtype=torch.float32, device=cuda)
    cache = torch.zeros(((k - 1) * d, c_in), dtype=torch.float32, device=cuda)
    rng = np.random.default_rng(7)
    for call in range(2):
        x = torch.tensor(rng.standard_normal((n, c_in)), dtype=torch.float32, device=cuda)
        y_ref = torch.empty((n, c_out), dtype=torch.float32, device=cuda)
        stream.process(x, y_ref)
        y = torch.full((n, c_out), float("nan"), dtype=torch.float32, device=cuda)
        api.cached_conv1d_static(x, wt, bt, cache, y, dilation=d, pad_left=half,
                                 pad_right=(k - 1) * d - half, act_in=act)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy().astype(np.float64)
        out = y.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(out))
        err = metrics.max_abs(ref, out)
        assert err <= FP32_TOL * metrics.rms(ref), f"call {call}: max-abs {err:.3e}"


def test_static_scratch_rejects_oversized_layer(cclib, cuda):
    import torch

    x = torch.zeros((4096, 1024), dtype=torch.float32, device=cuda)
    w = torch.zeros((1024, 1024, 3), dtype=torch.float32, device=cuda)
    cache = torch.zeros((2, 1024), dtype=torch.float32, device=cuda)
    y = torch.zeros((4096, 1024), dtype=torch.float32, device=cuda)
    with pytest.raises(api.CCError) as e:
        api.cached_conv1d_static(x, w, None, cache, y, dilation=1, pad_left=1, pad_right=1)
    assert e.value.status == -1 and "static scratch holds" in str(e.value)
