"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

FP32 bar: max |out - oracle| <= 1e-5 x RMS(oracle) on every compared sample.
Compared against the oracle's causal-offline model (which the oracle's own
streaming equals exactly, section 4.2) and against the original non-causal
model delayed by the computed latency on the interior."""
import numpy as np
import pytest

from oracle import metrics
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
LP_SNR_DB = 35.0
LP_MAXABS = 2e-2


def _assert_lowp(out, ref, what=""):
    """BF16 / FP16 bar: SNR >= 35 dB and max-abs <= 2e-2 x peak |ref|."""
    out = np.asarray(out, np.float64)
    ref = np.asarray(ref, np.float64)
    assert out.shape == ref.shape, (out.shape, ref.shape)
    snr = metrics.snr_db(ref, out)
    err = metrics.max_abs(ref, out)
    peak = float(np.max(np.abs(ref)))
    assert snr >= LP_SNR_DB, f"{what}: SNR {snr:.1f} dB < {LP_SNR_DB}"
    assert err <= LP_MAXABS * peak, f"{what}: max-abs {err:.3e} > {LP_MAXABS} x peak {peak:.3e}"
    return snr, err / peak


def _assert_fp32(out, ref, what=""):
    out = np.asarray(out, np.float64)
    ref = np.asarray(ref, np.float64)
    assert out.shape == ref.shape, (out.shape, ref.shape)
    err = metrics.max_abs(ref, out)
    bound = FP32_TOL * metrics.rms(ref)
    assert err <= bound, f"{what}: max-abs {err:.3e} > {bound:.3e} (rms {metrics.rms(ref):.3e})"


def _decoder(seed=1):
    dec = W.rave_decoder()
    p = W.init_params(dec, seed)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    return dec, p


def _encoder(seed=4):
    enc = W.rave_encoder()
    p = W.init_params(enc, seed)
    _, g, _, _ = pqmf.design(16, 64)
    p[W.pqmf_node_index(enc)] = (pqmf.analysis_weights(g), None)
    return enc, p


def _run_stream(model, stream, x, partition, torch, dev):
    outs, pos = [], 0
    io = model.io
    for n in partition:
        xb = torch.tensor(x[pos:pos + n], dtype=torch.float32, device=dev).contiguous()
        yb = torch.empty((n // io["in_per_step"] * io["out_per_step"], io["out_channels"]),
                         dtype=torch.float32, device=dev)
        stream.process(xb, yb)
        outs.append(yb.cpu().numpy())
        pos += n
    torch.cuda.synchronize()
    return np.concatenate(outs, axis=0)


def test_tiny_config_32_buffers_of_512(cclib, cuda):
    import torch

    nodes = W.tiny_stack()
    p = W.init_params(nodes, 0)
    x = W.signal(0, 16384, 16)
    model = api.Model(nodes, p, max_streams=2, max_steps_per_call=512)
    assert model.total_delay == 7
    s = model.stream(seed=0)
    y = _run_stream(model, s, x, [512] * 32, torch, cuda)
    yc = M.run_causal(nodes, p, x)
    _assert_fp32(y, yc, "tiny streamed vs causal offline")
    yo = M.run_original(nodes, p, x)
    d, w = 7, M.warmup_frames(nodes)
    _assert_fp32(y[d + w:], yo[w:len(yo) - d], "tiny streamed vs original delayed")


@pytest.mark.parametrize("partition,max_steps", [([1, 1, 1, 5, 64, 3, 437, 512, 1024, 2048], 512),
                                                 ([4096], 4096), ([3] * 40, 2)])
def test_tiny_ragged_buffers(cclib, cuda, partition, max_steps):
    import torch

    nodes = W.tiny_stack()
    p = W.init_params(nodes, 2)
    total = sum(partition)
    x = W.signal(3, total, 16)
    model = api.Model(nodes, p, max_streams=1, max_steps_per_call=max_steps)
    y = _run_stream(model, model.stream(), x, partition, torch, cuda)
    _assert_fp32(y, M.run_causal(nodes, p, x), f"tiny partition {partition[:4]}...")


def test_decoder_fp32_single_stream_full_length(cclib, cuda):
    """The decoder workload at full length: 235 latent frames (10 s at 48 kHz),
    one 2048-sample buffer per call, every output sample compared."""
    import torch

    dec, p = _decoder()
    frames = 235
    z = W.signal(1, frames, 128)
    model = api.Model(dec, p, max_streams=1, max_steps_per_call=1)
    assert model.total_delay == 12424
    s = model.stream(seed=11)
    y = _run_stream(model, s, z, [1] * frames, torch, cuda)
    yc = M.run_causal(dec, p, z, seed=11)
    _assert_fp32(y, yc, "decoder streamed vs causal offline")
    yo = M.run_original(dec, p, z, seed=11)
    d, w = 12424, M.warmup_frames(dec)
    _assert_fp32(y[d + w:], yo[w:len(yo) - d], "decoder vs original delayed")


def test_decoder_buffer_size_invariance(cclib, cuda):
    """Section 4.2: the streamed output does not depend on the buffer sizes."""
    import torch

    dec, p = _decoder(3)
    z = W.signal(7, 12, 128)
    yc = M.run_causal(dec, p, z, seed=5)
    for part, ms in (([2, 1, 3, 4, 2], 2), ([12], 4), ([5, 7], 3)):
        model = api.Model(dec, p, max_streams=1, max_steps_per_call=ms)
        y = _run_stream(model, model.stream(seed=5), z, part, torch, cuda)
        _assert_fp32(y, yc, f"decoder partition {part}")
        model.close()


def test_decoder_batched_streams_match_oracle_and_alone(cclib, cuda):
    import torch

    dec, p = _decoder(4)
    count, steps = 6, 5
    seeds = W.stream_seeds(21, count)
    zs = [W.signal(100 + i, steps, 128) for i in range(count)]
    model = api.Model(dec, p, max_streams=count + 1, max_steps_per_call=1)
    streams = [model.stream(seed=s) for s in seeds]
    outs = np.zeros((count, steps * 2048, 1))
    for t in range(steps):
        x = torch.tensor(np.stack([z[t:t + 1] for z in zs]), dtype=torch.float32, device=cuda)
        y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
        model.process_batch(streams, x, y)
        outs[:, t * 2048:(t + 1) * 2048] = y.cpu().numpy()
    alone = model.stream(seed=seeds[2])
    ya = _run_stream(model, alone, zs[2], [1] * steps, torch, cuda)
    for i in range(count):
        _assert_fp32(outs[i], M.run_causal(dec, p, zs[i], seed=seeds[i]), f"batched stream {i}")
    _assert_fp32(ya, outs[2], "alone vs in the batch")


def test_encoder_strided_and_pqmf_analysis(cclib, cuda):
    import torch

    enc, p = _encoder()
    x = W.signal(4, 2048 * 9, 1, std=0.1)
    model = api.Model(enc, p, max_streams=1, max_steps_per_call=2)
    assert model.total_delay == 3
    y = _run_stream(model, model.stream(), x, [2048, 4096, 2048 * 3, 2048 * 3], torch, cuda)
    yc = M.run_causal(enc, p, x)
    _assert_fp32(y, yc, "encoder streamed vs causal offline")


def test_checkpoint_resume_and_reset(cclib, cuda):
    import torch

    dec, p = _decoder(5)
    z = W.signal(9, 8, 128)
    model = api.Model(dec, p, max_streams=3, max_steps_per_call=2)
    a = model.stream(seed=3)
    first = _run_stream(model, a, z[:4], [2, 2], torch, cuda)
    blob = a.get_state()
    rest_a = _run_stream(model, a, z[4:], [1, 3], torch, cuda)
    b = model.stream(seed=999)
    b.set_state(blob)
    rest_b = _run_stream(model, b, z[4:], [2, 2], torch, cuda)
    _assert_fp32(rest_b, rest_a, "restored stream")
    a.reset()
    again = _run_stream(model, a, z[:4], [4], torch, cuda)
    _assert_fp32(again, first, "after reset")


def test_host_buffers_match_device_buffers(cclib, cuda):
    import torch

    nodes = W.tiny_stack()
    p = W.init_params(nodes, 6)
    x = W.signal(6, 2048, 16).astype(np.float32)
    model = api.Model(nodes, p, max_streams=2, max_steps_per_call=1024)
    s1, s2 = model.stream(), model.stream()
    yh = np.zeros((2048, 16), np.float32)
    s1.process(x, yh)
    torch.cuda.synchronize()
    yd = _run_stream(model, s2, x, [2048], torch, cuda)
    np.testing.assert_array_equal(yh, yd)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_host_buffer_batches_replay_one_graph(cclib, cuda, dtype):
    """Batched calls with host buffers run their launch chain from a CUDA graph
    captured on the first call (for that number of streams and steps) and
    replayed after; two groups of streams on two CUDA streams use staging of
    their own.  Every call equals, bit for bit, the same streams driven with
    device buffers."""
    import torch

    dec = W.rave_decoder(latent=16, capacity=16 if dtype == "f32" else 64, ratios=(2, 2), dilations=(1, 3),
                         bands=4, pqmf_taps=16)
    p = W.init_params(dec, 3)
    _, g, _, _ = pqmf.design(4, 16)
    p[W.pqmf_node_index(dec)] = (pqmf.synthesis_weights(g), None)
    steps, n = 6, 3
    z = np.random.default_rng(2).standard_normal((steps, 2 * n, 1, 16)).astype(np.float32)
    cs = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = {}
    for host in (True, False):
        model = api.Model(dec, p, dtype=dtype, max_streams=2 * n, max_steps_per_call=1)
        groups = [[model.stream(seed=10 * k + i) for i in range(n)] for k in range(2)]
        ops = model.io["out_per_step"]
        o = np.zeros((2 * n, steps * ops), np.float32)
        for t in range(steps):
            for k in range(2):
                zk = z[t, k * n:(k + 1) * n]
                if host:
                    y = np.zeros((n, ops, 1), np.float32)
                    model.process_batch(groups[k], np.ascontiguousarray(zk), y, cuda_stream=cs[k])
                    cs[k].synchronize()
                    o[k * n:(k + 1) * n, t * ops:(t + 1) * ops] = y[:, :, 0]
                else:
                    with torch.cuda.stream(cs[k]):
                        y = torch.empty((n, ops, 1), dtype=torch.float32, device=cuda)
                        model.process_batch(groups[k], torch.tensor(zk, device=cuda), y, cuda_stream=cs[k])
                    cs[k].synchronize()
                    o[k * n:(k + 1) * n, t * ops:(t + 1) * ops] = y[:, :, 0].cpu().numpy()
        assert model.device_status() == 0
        outs[host] = o
        model.close()
    np.testing.assert_array_equal(outs[True], outs[False])


def test_errors(cclib, cuda):
    import torch

    nodes = W.rave_encoder()
    p = W.init_params(nodes, 0)
    _, g, _, _ = pqmf.design(16, 64)
    p[1] = (pqmf.analysis_weights(g), None)
    model = api.Model(nodes, p, max_streams=1, max_steps_per_call=1)
    s = model.stream()
    with pytest.raises(api.CCError) as e:  # not a whole model step
        s.process(torch.zeros((1000, 1), device=cuda), torch.zeros((0, 128), device=cuda))
    assert e.value.status == -3
    with pytest.raises(api.CCError) as e:  # wrong output length
        s.process(torch.zeros((2048, 1), device=cuda), torch.zeros((2, 128), device=cuda))
    assert e.value.status == -3
    with pytest.raises(api.CCError) as e:  # arena full: admission by cache memory
        model.stream()
    assert e.value.status == -4
    s.close()
    model.stream().close()  # the slot came back
    # empty buffers are a no-op
    s2 = model.stream()
    s2.process(torch.zeros((0, 1), device=cuda), torch.zeros((0, 128), device=cuda))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_decoder_full_batch_sampled_streams(cclib, cuda, dtype):
    """The benchmark's launch configuration (256 streams x one 2048-sample
    buffer per step, max one step per call): every stream runs on the GPU,
    a sample of streams is checked sample-by-sample against the oracle, over
    24 steps: every ring of the model wraps (the longest, a low-precision view
    of stage 0, holds 18 steps)."""
    import torch

    dec, p = _decoder(1)
    count, steps = 256, 24
    seeds = W.stream_seeds(1000, count)
    z = np.random.default_rng(0).standard_normal((steps, count, 1, 128))
    model = api.Model(dec, p, dtype=dtype, max_streams=count, max_steps_per_call=1)
    streams = [model.stream(seed=s) for s in seeds]
    y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
    outs = np.zeros((count, steps * 2048))
    for t in range(steps):
        model.process_batch(streams, torch.tensor(z[t], dtype=torch.float32, device=cuda), y)
        outs[:, t * 2048:(t + 1) * 2048] = y[:, :, 0].cpu().numpy()
    assert model.device_status() == 0
    for i in (0, 77, 200, 255):
        ref = M.run_causal(dec, p, z[:, i, 0, :], seed=seeds[i])[:, 0]
        if dtype == "f32":
            _assert_fp32(outs[i], ref, f"stream {i} of {count}")
        else:
            _assert_lowp(outs[i], ref, f"{dtype} stream {i} of {count}")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_decoder_lowp_single_stream_partitions(cclib, cuda, dtype):
    """Tensor-core path with one stream (partial tiles everywhere) and ragged
    buffers; per-buffer-size invariance within the precision bar."""
    import torch

    dec, p = _decoder(6)
    z = W.signal(8, 10, 128)
    ref = M.run_causal(dec, p, z, seed=4)
    for part, ms in (([1] * 10, 1), ([3, 2, 5], 3)):
        model = api.Model(dec, p, dtype=dtype, max_streams=1, max_steps_per_call=ms)
        y = _run_stream(model, model.stream(seed=4), z, part, torch, cuda)
        assert model.device_status() == 0
        _assert_lowp(y, ref, f"{dtype} partition {part}")
        model.close()


def test_decoder_bf16_noise_off_vs_original(cclib, cuda):
    """Section 4.2 setting (noise synthesiser off): BF16 streamed output vs the
    original non-causal model, delayed by the computed latency."""
    import torch

    dec, p = _decoder(7)
    z = W.signal(9, 16, 128)
    model = api.Model(dec, p, dtype="bf16", max_streams=1, max_steps_per_call=2, noise=False)
    y = _run_stream(model, model.stream(seed=1), z, [2] * 8, torch, cuda)
    yo = M.run_original(dec, p, z, seed=1, noise_on=False)
    d, w = model.total_delay, M.warmup_frames(dec)
    _assert_lowp(y[d + w:], yo[w:len(yo) - d], "bf16 vs original delayed")


def test_lowp_window_boxes_match_gathers(cclib, cuda):
    """The tensor-core producer loads a tile's window rows as one 3D box when
    its streams sit in consecutive slots at one step, and gathers them row by
    row otherwise.  Both forms feed the same operands to the same MMAs, so a
    batch in slot order (boxes, a partial last tile whose box reaches past the
    last slot) and the same streams in reverse order (gathers) agree exactly,
    over enough steps for every ring to wrap through its mirrored tail; one
    stream is checked against the oracle."""
    import torch

    dec, p = _decoder(11)
    count, steps = 50, 40
    seeds = W.stream_seeds(77, count)
    z = np.random.default_rng(5).standard_normal((steps, count, 1, 128))
    outs = []
    for order in (np.arange(count), np.arange(count)[::-1]):
        model = api.Model(dec, p, dtype="bf16", max_streams=count, max_steps_per_call=1)
        streams = [model.stream(seed=s) for s in seeds]
        batch = [streams[i] for i in order]
        y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
        o = np.zeros((count, steps * 2048))
        for t in range(steps):
            model.process_batch(batch, torch.tensor(z[t][order], dtype=torch.float32, device=cuda), y)
            o[order, t * 2048:(t + 1) * 2048] = y[:, :, 0].cpu().numpy()
        assert model.device_status() == 0
        outs.append(o)
        model.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = M.run_causal(dec, p, z[:, 31, 0, :], seed=seeds[31])[:, 0]
    _assert_lowp(outs[0][31], ref, "bf16 stream 31 of 50, 40 steps")


@pytest.mark.parametrize("count,dtype", [(256, "bf16"), (250, "bf16"), (250, "f16")])
def test_fused_residual_units_equal_unfused(cclib, cuda, count, dtype):
    """A residual unit (k=3 conv -> 1x1 conv + skip) runs as one tensor-core
    launch, its intermediate rounded to BF16 in shared memory exactly as the
    unfused path rounds it into its ring: up to 128 channels in one CTA, the
    decoder's 256-channel stage-1 units as clusters of two CTAs that exchange
    their halves of the intermediate in distributed shared memory (the
    unfused model then runs those layers unsplit, so both sum in one order).
    The two give identical outputs with fewer launches fused.  One stream is
    also checked against the oracle."""
    import torch

    dec, p = _decoder(12)
    steps = 4
    seeds = W.stream_seeds(21, count)
    z = np.random.default_rng(6).standard_normal((steps, count, 1, 128))
    outs, launches = [], []
    for fuse in (True, False):
        model = api.Model(dec, p, dtype=dtype, max_streams=count, max_steps_per_call=1, fuse_units=fuse)
        streams = [model.stream(seed=s) for s in seeds]
        y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
        o = np.zeros((count, steps * 2048))
        for t in range(steps):
            model.process_batch(streams, torch.tensor(z[t], dtype=torch.float32, device=cuda), y)
            o[:, t * 2048:(t + 1) * 2048] = y[:, :, 0].cpu().numpy()
        assert model.device_status() == 0
        outs.append(o)
        launches.append(model.chain_launches)
        model.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    # the three residual units of each of stages 1, 2 and 3 are one launch each
    # fused (stage 0, 512 channels, stays unfused)
    assert launches[0] == launches[1] - 9, launches
    k = count // 3
    ref = M.run_causal(dec, p, z[:, k, 0, :], seed=seeds[k])[:, 0]
    _assert_lowp(outs[0][k], ref, f"{dtype} fused units, stream {k} of {count}")


def test_merged_sibling_convs_equal_separate(cclib, cuda):
    """The decoder's three head convolutions (k = 7, 3, 3, all reading
    LeakyReLU(h)) run as one tensor-core contraction with right-aligned
    windows (zero taps in front of the shorter kernels) and their FP32 outputs
    side by side in one ring; adding exact zeros leaves every sum unchanged,
    so the outputs equal those of three separate launches.  Checked with a
    partial last tile (250 streams) and against the oracle for one stream."""
    import torch

    dec, p = _decoder(13)
    count, steps = 250, 4
    seeds = W.stream_seeds(31, count)
    z = np.random.default_rng(7).standard_normal((steps, count, 1, 128))
    outs = []
    for merge in (True, False):
        model = api.Model(dec, p, dtype="bf16", max_streams=count, max_steps_per_call=1, merge_siblings=merge)
        streams = [model.stream(seed=s) for s in seeds]
        y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
        o = np.zeros((count, steps * 2048))
        for t in range(steps):
            model.process_batch(streams, torch.tensor(z[t], dtype=torch.float32, device=cuda), y)
            o[:, t * 2048:(t + 1) * 2048] = y[:, :, 0].cpu().numpy()
        assert model.device_status() == 0
        outs.append(o)
        model.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = M.run_causal(dec, p, z[:, 99, 0, :], seed=seeds[99])[:, 0]
    _assert_lowp(outs[0][99], ref, "bf16 merged heads, stream 99 of 250")
