"""The stream-local tail kernel (cc_kernels_tail.cu): the suffix of the launch
chain whose layers read only their own streams' frames runs as one
persistent kernel in which each CTA takes a group of streams through every
layer (transposed tcgen05 contractions, fused residual units, narrow FP32
convolutions, the heads merge and the inverse PQMF).  It must meet the
low-precision bar against the oracle and agree closely with the same model
launched layer by layer, at the benchmark's 256 streams and with groups that
leave partial tiles (odd stream counts), over enough steps for every ring of
the tail to wrap."""
import numpy as np
import pytest

from oracle import metrics
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _decoder(seed=1):
    dec = W.rave_decoder()
    p = W.init_params(dec, seed)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    return dec, p


def _run(model, streams, z, cuda):
    import torch

    count, steps = z.shape[1], z.shape[0]
    y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
    outs = np.zeros((count, steps * 2048))
    for t in range(steps):
        model.process_batch(streams, torch.tensor(z[t], dtype=torch.float32, device=cuda), y)
        outs[:, t * 2048:(t + 1) * 2048] = y[:, :, 0].cpu().numpy()
    assert model.device_status() == 0
    return outs


@pytest.mark.parametrize("count", [256, 37])
def test_tail_kernel_matches_layer_by_layer_and_oracle(cclib, cuda, count):
    dec, p = _decoder(3)
    steps = 12
    seeds = W.stream_seeds(500, count)
    z = np.random.default_rng(count).standard_normal((steps, count, 1, 128))
    outs = {}
    for tail in (True, False):
        model = api.Model(dec, p, dtype="bf16", max_streams=count, max_steps_per_call=1, tail_fusion=tail)
        streams = [model.stream(seed=s) for s in seeds]
        outs[tail] = _run(model, streams, z, cuda)
        model.close()
    for i in sorted({0, count // 2, count - 1}):
        ref = M.run_causal(dec, p, z[:, i, 0, :], seed=seeds[i])[:, 0]
        for tail in (True, False):
            snr = metrics.snr_db(ref, outs[tail][i])
            err = metrics.max_abs(ref, outs[tail][i])
            assert snr >= 35.0 and err <= 2e-2 * np.max(np.abs(ref)), f"tail={tail} stream {i}: {snr:.1f} dB"
    agree = min(metrics.snr_db(outs[False][i], outs[True][i]) for i in range(count))
    assert agree >= 60.0, f"tail vs layer-by-layer: {agree:.1f} dB"
