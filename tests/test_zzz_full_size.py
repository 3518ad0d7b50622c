"""Full and maximum sizes.

* Parity at the launch configuration bench.py times for the audio -> audio
  workload (autoencoder-bf16-b256): the RAVE-like encoder feeding the decoder,
  BF16, a model of 256 streams, every call one 2048-sample buffer for all 256
  streams.  Sampled streams are checked sample by sample against the FP64
  oracle at the BF16 bar (SNR >= 35 dB, max-abs <= 2e-2 x peak).
* The largest arena: the tensor-core epilogue addresses the arena with 32-bit
  offsets in 16-byte units, so a model whose arena would reach 64 GiB is
  refused with CC_ERR_NO_MEMORY before the arena is allocated, and one just
  below the limit is accepted.

The file runs after every other test, so that a failure here never hides
another test's result."""
import numpy as np
import pytest

from oracle import metrics
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autoencoder_bf16_256_streams_sampled(cclib, cuda):
    import torch

    enc, dec = W.rave_encoder(), W.rave_decoder()
    nodes = W.chain(enc, dec)
    p = W.init_params(nodes, 1)
    _, g, _, _ = pqmf.design(16, 64)
    for i, nd in enumerate(nodes):
        if nd["name"] == "pqmf":
            p[i] = (pqmf.analysis_weights(g), None)
        if nd["name"] == "ipqmf":
            p[i] = (pqmf.synthesis_weights(g), None)
    count, T = 256, 3
    seeds = W.stream_seeds(1000, count)
    xs = np.stack([W.signal(700 + i, 2048 * T, 1, std=0.1) for i in range(count)])
    model = api.Model(nodes, p, dtype="bf16", max_streams=count, max_steps_per_call=1)
    streams = [model.stream(seed=s) for s in seeds]
    y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
    outs = []
    for t in range(T):
        x = torch.tensor(xs[:, 2048 * t:2048 * (t + 1)], dtype=torch.float32, device=cuda)
        model.process_batch(streams, x, y)
        outs.append(y.cpu().numpy())
    torch.cuda.synchronize()
    model.device_status()
    out = np.concatenate(outs, axis=1)[:, :, 0]
    for i in (0, 77, 128, 255):
        ref = M.run_causal(nodes, p, xs[i], seed=seeds[i])[:, 0]
        snr, err, peak = metrics.snr_db(ref, out[i]), metrics.max_abs(ref, out[i]), float(np.max(np.abs(ref)))
        print(f"stream {i}: SNR {snr:.1f} dB, max-abs / peak {err / peak:.2e}")
        assert snr >= 35.0, f"stream {i}: SNR {snr:.1f} dB"
        assert err <= 2e-2 * peak, f"stream {i}: max-abs {err:.3e} > 2e-2 x {peak:.3e}"
    model.close()


def test_arena_limit_of_64_gib(cclib, cuda):
    dec = W.rave_decoder()
    p = W.init_params(dec, 1)
    slot = api.Model(dec, {}, dtype="bf16", max_streams=0).state_bytes[1]
    too_many = (1 << 36) // slot + 1
    assert too_many * slot >= 1 << 36
    with pytest.raises(api.CCError) as e:
        api.Model(dec, p, dtype="bf16", max_streams=too_many)
    assert e.value.status == -4
    # just below the limit the arena is taken (about 64 GB of the GPU's 288)
    m = api.Model(dec, p, dtype="bf16", max_streams=too_many - 1)
    s = m.stream(seed=1)
    s.close()
    m.close()
