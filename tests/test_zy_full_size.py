"""Full and maximum sizes.

* Parity at the launch configuration bench.py times for the audio -> audio
  workload (autoencoder-bf16-b256): the RAVE-like encoder feeding the decoder,
  BF16, a model of 256 streams, every call one 2048-sample buffer for all 256
  streams.  Sampled streams are checked sample by sample against the FP64
  oracle at the BF16 bar (SNR >= 35 dB, max-abs <= 2e-2 x peak).
* The largest arena: the tensor-core epilogue addresses the arena with 32-bit
  offsets in 16-byte units, so a model whose arena would reach 64 GiB is
  refused with CC_ERR_NO_MEMORY before the arena is allocated; in the largest
  model allowed, the stream in the top slot computes bit for bit what the
  stream in slot 0 computes.

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
    import torch

    dec = W.rave_decoder()
    p = W.init_params(dec, 1)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    slot = api.Model(dec, {}, dtype="bf16", max_streams=0).state_bytes[1]
    too_many = (1 << 36) // slot + 1
    assert too_many * slot >= 1 << 36 > (too_many - 1) * slot
    with pytest.raises(api.CCError) as e:
        api.Model(dec, p, dtype="bf16", max_streams=too_many)
    assert e.value.status == -4
    # the largest model allowed (about 64 GB of arena): every slot taken, so
    # the last stream sits in the top slot, whose 16-byte offsets come within
    # one slot of 2^32; it computes exactly what slot 0 computes, batched with
    # it (row gathers) and alone (window boxes)
    n = too_many - 1
    m = api.Model(dec, p, dtype="bf16", max_streams=n, max_steps_per_call=1)
    streams = [m.stream(seed=7) for _ in range(n)]  # slots 0 .. n - 1 in order
    first, last = streams[0], streams[-1]
    z = W.signal(3, 3, 128)
    y2 = torch.empty((2, 2048, 1), dtype=torch.float32, device=cuda)
    y1 = torch.empty((1, 2048, 1), dtype=torch.float32, device=cuda)
    x2 = torch.tensor(np.stack([z[0:1], z[0:1]]), dtype=torch.float32, device=cuda)
    m.process_batch([first, last], x2, y2)
    out = y2.cpu().numpy()
    assert np.array_equal(out[0], out[1])
    for t in (1, 2):
        x1 = torch.tensor(z[None, t:t + 1], dtype=torch.float32, device=cuda)
        m.process_batch([first], x1, y1)
        a = y1.cpu().numpy().copy()
        m.process_batch([last], x1, y1)
        assert np.array_equal(a, y1.cpu().numpy())
    torch.cuda.synchronize()
    m.device_status()
    m.close()
