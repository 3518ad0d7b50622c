"""The C-ABI calls around the per-buffer DSP call (section 1, section 5.1):
ragged batches (cc_process_batch), buffers that are not whole model steps
(FIFO mode, cc_stream_set_fifo / cc_stream_delay) and admission by cache
memory (cc_model_config.arena_bytes, cc_model_capacity).  Outputs are
compared with the FP64 oracle's causal model, delayed by the stream's
reported latency (section 4.2)."""
import math

import numpy as np
import pytest

from oracle import metrics
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _small_decoder(seed=1):
    nodes = W.rave_decoder(latent=16, capacity=16, ratios=(4, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    p = W.init_params(nodes, seed)
    _, g, _, _ = pqmf.design(4, 16)
    p[W.pqmf_node_index(nodes)] = (pqmf.synthesis_weights(g), None)
    return nodes, p


def _small_chain(seed=2):
    enc = W.rave_encoder(latent=16, capacity=8, ratios=(2, 2), bands=4, pqmf_taps=16)
    dec = W.rave_decoder(latent=16, capacity=8, ratios=(2, 2), dilations=(1, 3), bands=4, pqmf_taps=16)
    nodes = W.chain(enc, dec)
    p = W.init_params(nodes, seed)
    _, g, _, _ = pqmf.design(4, 16)
    for i, nd in enumerate(nodes):
        if nd["name"] == "pqmf":
            p[i] = (pqmf.analysis_weights(g), None)
        if nd["name"] == "ipqmf":
            p[i] = (pqmf.synthesis_weights(g), None)
    return nodes, p


def _check(ref, out):
    err = metrics.max_abs(ref, out)
    assert err <= FP32_TOL * metrics.rms(ref), f"max-abs {err:.3e} > {FP32_TOL} x rms {metrics.rms(ref):.3e}"


def test_ragged_batch_matches_oracle(cclib, cuda):
    """Streams advanced by different numbers of whole steps in one call (zero
    included), host and device buffers mixed, over several calls."""
    import torch

    nodes, p = _small_decoder()
    model = api.Model(nodes, p, max_streams=5, max_steps_per_call=2)
    io = model.io
    seeds = [11, 12, 13, 14, 15]
    streams = [model.stream(seed=s) for s in seeds]
    calls = [[1, 0, 3, 2, 1], [2, 2, 0, 1, 4], [0, 1, 1, 0, 2]]  # steps per stream per call
    total = [sum(c[i] for c in calls) for i in range(5)]
    z = [W.signal(40 + i, total[i], io["in_channels"]) for i in range(5)]
    outs = [[] for _ in range(5)]
    pos = [0] * 5
    for ci, steps in enumerate(calls):
        xs, ys = [], []
        for i, k in enumerate(steps):
            if k == 0:
                xs.append(None)
                ys.append(None)
                continue
            x = z[i][pos[i]:pos[i] + k].astype(np.float32)
            if (i + ci) % 2:  # device buffers for some, host for the others
                xs.append(torch.tensor(x, device=cuda))
                ys.append(torch.full((k * io["out_per_step"], 1), float("nan"), device=cuda))
            else:
                xs.append(np.ascontiguousarray(x))
                ys.append(np.full((k * io["out_per_step"], 1), np.nan, np.float32))
            pos[i] += k
        model.process_ragged(streams, xs, ys)
        torch.cuda.synchronize()
        for i, y in enumerate(ys):
            if y is not None:
                outs[i].append(y.cpu().numpy() if hasattr(y, "cpu") else y.copy())
    for i in range(5):
        ref = M.run_causal(nodes, p, z[i], seed=seeds[i])
        _check(ref, np.concatenate(outs[i]).astype(np.float64))


def test_ragged_batch_rejects_bad_lengths_and_duplicates(cclib, cuda):
    nodes, p = _small_decoder()
    model = api.Model(nodes, p, max_streams=2, max_steps_per_call=1)
    a, b = model.stream(), model.stream()
    ops = model.io["out_per_step"]
    x = np.zeros((1, 16), np.float32)
    with pytest.raises(api.CCError) as e:
        model.process_ragged([a, b], [x, x], [np.zeros((ops, 1), np.float32), np.zeros((ops - 1, 1), np.float32)])
    assert e.value.status == -3
    with pytest.raises(api.CCError) as e:
        model.process_ragged([a, a], [x, x], [np.zeros((ops, 1), np.float32)] * 2)
    assert e.value.status == -1


def test_fifo_decoder_sub_step_buffers(cclib, cuda):
    """A decoder whose model step emits 32 samples, asked for 8-sample buffers:
    each step's latent frame comes with the first call that needs its output,
    so no prefill is needed and the delay is the model's."""
    import torch

    nodes, p = _small_decoder()
    model = api.Model(nodes, p, max_streams=1, max_steps_per_call=1)
    ops = model.io["out_per_step"]
    assert ops == 32
    s = model.stream(seed=5)
    s.set_fifo(True, prefill=0)
    assert s.delay == model.total_delay
    frames = 6
    z = W.signal(9, frames, 16)
    outs, sent, asked = [], 0, 0
    for b in [8] * (frames * ops // 8):
        asked += b
        need = -(-asked // ops)
        x = torch.tensor(z[sent:need], dtype=torch.float32, device=cuda).reshape(need - sent, 16)
        y = torch.empty((b, 1), dtype=torch.float32, device=cuda)
        s.process(x, y)
        sent = need
        outs.append(y.cpu().numpy())
    ref = M.run_causal(nodes, p, z, seed=5)
    _check(ref, np.concatenate(outs).astype(np.float64))
    assert s.fifo_state == (0, 0)
    # asking for output whose input has not come is refused, with nothing changed
    y = torch.empty((8, 1), dtype=torch.float32, device=cuda)
    with pytest.raises(api.CCError) as e:
        s.process(torch.empty((0, 16), dtype=torch.float32, device=cuda), y)
    assert e.value.status == -3
    assert s.fifo_state == (0, 0)


@pytest.mark.parametrize("b", [4, 6])
def test_fifo_audio_to_audio_fixed_buffers(cclib, cuda, b):
    """Encoder -> decoder (a step is 16 samples in and out) called with b-sample
    buffers in and out: prefill = 16 - gcd(b, 16) zero samples make every call
    servable, and the stream's delay grows by exactly that (reading R5).  After
    a reset the stream starts over."""
    import torch

    nodes, p = _small_chain()
    model = api.Model(nodes, p, max_streams=1, max_steps_per_call=2)
    io = model.io
    assert io["in_per_step"] == 16 and io["out_per_step"] == 16
    pre = 16 - math.gcd(b, 16)
    s = model.stream(seed=3)
    s.set_fifo(True, prefill=pre)
    assert s.delay == model.total_delay + pre
    n = 16 * 12
    x = W.signal(8, n, 1, std=0.1)
    ref = np.concatenate([np.zeros((pre, 1)), M.run_causal(nodes, p, x, seed=3)])[:n]
    for attempt in range(2):
        outs = []
        for t in range(0, n, b):
            xb = torch.tensor(x[t:t + b], dtype=torch.float32, device=cuda)
            yb = torch.empty((xb.shape[0], 1), dtype=torch.float32, device=cuda)
            s.process(xb, yb)
            outs.append(yb.cpu().numpy())
        _check(ref, np.concatenate(outs).astype(np.float64))
        s.reset()
    s.set_fifo(False)
    assert s.delay == model.total_delay


def test_admission_by_arena_bytes(cclib, cuda):
    nodes, p = _small_decoder()
    plan = api.Model(nodes, p, max_streams=0)
    slot = plan.state_bytes[1]
    m = api.Model(nodes, p, max_streams=0, arena_bytes=int(3.5 * slot))
    assert m.capacity == (3, 3)
    ss = [m.stream(seed=i) for i in range(3)]
    assert m.capacity == (3, 0)
    with pytest.raises(api.CCError) as e:
        m.stream()
    assert e.value.status == -4
    ss[0].close()
    assert m.capacity == (3, 1)
    m.stream()
    capped = api.Model(nodes, p, max_streams=2, arena_bytes=10 * slot)
    assert capped.capacity == (2, 2)
    with pytest.raises(api.CCError) as e:
        api.Model(nodes, p, max_streams=0, arena_bytes=slot - 1)
    assert e.value.status == -4
