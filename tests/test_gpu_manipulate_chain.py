"""GPU parity of latent manipulation (sections 5.1 and 5.2) and of audio -> audio
streaming (the encoder feeding the decoder, section 5.1's `forward`), through
the C ABI against the FP64 oracle.

Bars: FP32 max |out - oracle| <= 1e-5 x RMS(oracle); BF16 SNR >= 35 dB and
max-abs <= 2e-2 x peak |oracle|."""
import numpy as np
import pytest

from oracle import manipulate as MP
from oracle import metrics
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _assert_fp32(out, ref, what=""):
    out, ref = np.asarray(out, np.float64), np.asarray(ref, np.float64)
    assert out.shape == ref.shape, (out.shape, ref.shape)
    err, bound = metrics.max_abs(ref, out), 1e-5 * metrics.rms(ref)
    assert err <= bound, f"{what}: max-abs {err:.3e} > {bound:.3e}"


def _assert_lowp(out, ref, what=""):
    out, ref = np.asarray(out, np.float64), np.asarray(ref, np.float64)
    assert out.shape == ref.shape, (out.shape, ref.shape)
    snr, err, peak = metrics.snr_db(ref, out), metrics.max_abs(ref, out), float(np.max(np.abs(ref)))
    print(f"{what}: SNR {snr:.1f} dB, max-abs / peak {err / peak:.2e}")
    assert snr >= 35.0, f"{what}: SNR {snr:.1f} dB"
    assert err <= 2e-2 * peak, f"{what}: max-abs {err:.3e} > 2e-2 x {peak:.3e}"


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


def _autoencoder(seed=6):
    """The encoder feeding the decoder as one model, and the same weights as
    two models (params are {node index: (w, b)})."""
    enc, dec = W.rave_encoder(), W.rave_decoder()
    nodes = W.chain(enc, dec)
    p = W.init_params(nodes, seed)
    _, g, _, _ = pqmf.design(16, 64)
    for i, nd in enumerate(nodes):
        if nd["name"] == "pqmf":
            p[i] = (pqmf.analysis_weights(g), None)
        if nd["name"] == "ipqmf":
            p[i] = (pqmf.synthesis_weights(g), None)
    off = len(enc) - 1  # decoder node k >= 1 is chain node off + k
    pe = {i: p[i] for i in range(len(enc)) if i in p}
    pd = {k: p[off + k] for k in range(1, len(dec)) if off + k in p}
    return nodes, p, (enc, pe), (dec, pd)


def _process(stream, x, n_out_per_in, torch, dev):
    xb = torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device=dev)
    yb = torch.empty((x.shape[0] * n_out_per_in[0] // n_out_per_in[1], 1), dtype=torch.float32, device=dev)
    stream.process(xb, yb)
    return yb


# ---------------------------------------------------------------- manipulation

def _controls(T, C):
    """Controls that change at frames 3, 6 and 9: Fig. 7's bias of the first
    dimension and replacement of the last one, then section 5.2's scale and
    noise on some dimensions, then back to the identity."""
    b1 = np.zeros(C)
    b1[0], b1[-1] = 1.5, -0.7
    s1 = np.ones(C)
    s1[-1] = 0.0
    s2 = s1.copy()
    s2[:C // 2] = 0.5
    a2 = np.zeros(C)
    a2[10:20] = 0.3
    scale = MP.piecewise(T, C, [(3, s1), (6, s2), (9, 1.0)], 1.0)
    bias = MP.piecewise(T, C, [(3, b1), (9, 0.0)], 0.0)
    amp = MP.piecewise(T, C, [(6, a2), (9, 0.0)], 0.0)
    return scale, bias, amp


def test_manipulation_decoder_fp32_changes_between_buffers(cclib, cuda):
    import torch

    dec, p = _decoder(1)
    T, C, seed = 12, 128, 31
    z = W.signal(8, T, C)
    scale, bias, amp = _controls(T, C)
    model = api.Model(dec, p, max_streams=1, max_steps_per_call=3)
    s = model.stream(seed=seed)
    outs, pos = [], 0
    for n in (1, 2, 3, 3, 1, 2):  # buffer edges at 1, 3, 6, 9, 10
        s.set_input_manipulation(scale[pos], bias[pos], amp[pos])
        outs.append(_process(s, z[pos:pos + n], (2048, 1), torch, cuda).cpu().numpy())
        pos += n
    zm = MP.manipulate(z, scale, bias, amp, seed=seed)
    _assert_fp32(np.concatenate(outs), M.run_causal(dec, p, zm, seed=seed), "manipulated decoder")
    model.close()


def test_manipulation_batched_bf16_per_stream(cclib, cuda):
    """250 streams, each with its own controls (some none): the manipulated
    streams meet the BF16 bar against the oracle; the streams left at the
    identity, and a manipulated stream after reset, give the same bits as in a
    batch where nothing is manipulated."""
    import torch

    dec, p = _decoder(2)
    count, T, C = 250, 4, 128
    seeds = W.stream_seeds(40, count)
    zs = np.stack([W.signal(500 + i, T, C) for i in range(count)])
    model = api.Model(dec, p, dtype="bf16", max_streams=count, max_steps_per_call=1)

    def ctl(i):
        b = np.zeros(C, np.float32)
        b[i % C] = 0.25 * (i % 7 - 3)
        return np.ones(C, np.float32), b, np.full(C, 0.2 if i % 2 == 0 else 0.0, np.float32)

    def run(streams):
        y = torch.empty((count, 2048, 1), dtype=torch.float32, device=cuda)
        out = []
        for t in range(T):
            x = torch.tensor(zs[:, t:t + 1], dtype=torch.float32, device=cuda)
            model.process_batch(streams, x, y)
            out.append(y.cpu().numpy())
        torch.cuda.synchronize()
        return np.concatenate(out, axis=1)[:, :, 0]

    plain = [model.stream(seed=s) for s in seeds]
    y_plain = run(plain)
    for s in plain:
        s.close()
    manip = [model.stream(seed=s) for s in seeds]
    for i, s in enumerate(manip):
        if i % 5:
            s.set_input_manipulation(*ctl(i))
    y_manip = run(manip)
    ident = [i for i in range(count) if i % 5 == 0]
    assert np.array_equal(y_manip[ident], y_plain[ident])
    for i in (1, 2, 123, 249):
        sc, b, a = ctl(i)
        zm = MP.manipulate(zs[i], sc, b, a, seed=seeds[i])
        _assert_lowp(y_manip[i], M.run_causal(dec, p, zm, seed=seeds[i])[:, 0], f"stream {i}")
    assert not np.allclose(y_manip[1], y_plain[1])
    for s in manip:
        s.reset()
    assert np.array_equal(run(manip), y_plain)
    model.close()


def test_manipulation_rejected_where_it_must_be(cclib, cuda):
    dec, p = _decoder(3)
    model = api.Model(dec, p, max_streams=1, max_steps_per_call=1)
    s = model.stream()
    with pytest.raises(api.CCError):  # wrong channel count
        api._check(api.lib().cc_stream_set_input_manipulation(s.handle, None, None, None, 64, None))
    with pytest.raises(api.CCError):  # non-finite control
        s.set_input_manipulation(bias=np.full(128, np.nan))
    # the hand-written backward refuses a manipulated stream (CC_ERR_STATE)
    grads = api.Grads(model, p)
    s.set_input_manipulation(bias=0.5)
    with pytest.raises(api.CCError) as e:
        grads.begin([s])
    assert e.value.status == -7
    s.set_input_manipulation()  # back to the identity: accepted again
    grads.begin([s])
    grads.close()
    model.close()


# ---------------------------------------------------------------- audio -> audio

def test_audio_to_audio_chain_fp32(cclib, cuda):
    import torch

    nodes, p, (enc, _), (dec, _) = _autoencoder(6)
    model = api.Model(nodes, p, max_streams=1, max_steps_per_call=3)
    assert model.total_delay == M.analyze(nodes)["delay"] == 3 * 2048 + M.analyze(dec)["delay"]
    x = W.signal(9, 2048 * 8, 1, std=0.1)
    s = model.stream(seed=12)
    outs, pos = [], 0
    for n in (2048, 4096, 2048, 6144, 2048):
        outs.append(_process(s, x[pos:pos + n], (1, 1), torch, cuda).cpu().numpy())
        pos += n
    _assert_fp32(np.concatenate(outs), M.run_causal(nodes, p, x, seed=12), "audio -> audio")
    model.close()


def test_encode_manipulate_decode_two_models_fp32(cclib, cuda):
    """The encode / decode pattern of section 5.1: two streamed models with the
    latent between them on the device and the decoder stream manipulated;
    equals the oracle's offline encoder, the manipulation, and the offline
    decoder, one after the other."""
    import torch

    _, _, (enc, pe), (dec, pd) = _autoencoder(8)
    me = api.Model(enc, pe, max_streams=1, max_steps_per_call=1)
    md = api.Model(dec, pd, max_streams=1, max_steps_per_call=1)
    se, sd = me.stream(), md.stream(seed=14)
    T = 9
    x = W.signal(10, 2048 * T, 1, std=0.1)
    scale, bias, amp = _controls(T, 128)
    outs = []
    for t in range(T):
        xb = torch.tensor(x[2048 * t:2048 * (t + 1)], dtype=torch.float32, device=cuda)
        zl = torch.empty((1, 128), dtype=torch.float32, device=cuda)
        se.process(xb, zl)
        sd.set_input_manipulation(scale[t], bias[t], amp[t])
        y = torch.empty((2048, 1), dtype=torch.float32, device=cuda)
        sd.process(zl, y)
        outs.append(y.cpu().numpy())
    zc = M.run_causal(enc, pe, x)
    ref = M.run_causal(dec, pd, MP.manipulate(zc, scale, bias, amp, seed=14), seed=14)
    _assert_fp32(np.concatenate(outs), ref, "encode -> manipulate -> decode")
    me.close()
    md.close()


def _submit_audio(server, stream, x, buffers, tag0, keep):
    """One stream's requests: each gives b input samples and asks b output
    samples (a request shorter than the 2048-sample model step completes once
    the step's input is complete).  The output buffers go to `keep`: the
    scheduler thread writes them until their tags complete."""
    outs, tags, pos = [], [], 0
    for i, b in enumerate(buffers):
        out = np.zeros((b, 1), np.float32)
        keep.append(out)
        outs.append(out)
        tags.append(tag0 + i)
        server.submit([stream], [np.ascontiguousarray(x[pos:pos + b], dtype=np.float32)], [b], [out], [b],
                      [tag0 + i])
        pos += b
    return outs, tags


def _wait(server, tags, done):
    import time

    t0 = time.time()
    while not all(t in done for t in tags):
        got, _, _ = server.poll()
        done.update(int(t) for t in got)
        assert time.time() - t0 < 60, "requests not completed"
        time.sleep(0.001)


def test_audio_to_audio_served_bf16(cclib, cuda):
    """The audio -> audio model in the serving loop: a stream served alone with
    2048-sample buffers, and the same stream served with 512 / 1024 / 4096
    buffers among other streams, give the same output, which meets the BF16
    bar against the oracle."""
    nodes, p, _, _ = _autoencoder(10)
    model = api.Model(nodes, p, dtype="bf16", max_streams=6, max_steps_per_call=1)
    server = api.Server(model, max_batch=4, bucket=2)
    T = 6
    x = W.signal(11, 2048 * T, 1, std=0.1)
    keep, done = [], set()
    a = model.stream(seed=3)
    outs_a, tags_a = _submit_audio(server, a, x, [2048] * T, 7_000_000, keep)
    _wait(server, tags_a, done)
    server.remove(a)
    b = model.stream(seed=3)
    others = [model.stream(seed=50 + k) for k in range(2)]
    tags_o = []
    for k, s in enumerate(others):
        xo = W.signal(12 + k, 2048 * T, 1, std=0.1)
        tags_o += _submit_audio(server, s, xo, [4096, 2048, 4096, 2048], 7_100_000 + 100 * k, keep)[1]
    outs_b, tags_b = _submit_audio(server, b, x, [512, 1024, 512, 4096, 2048, 1024, 1024, 2048], 7_200_000, keep)
    _wait(server, tags_b + tags_o, done)
    ya = np.concatenate(outs_a)[:, 0]
    yb = np.concatenate(outs_b)[:, 0]
    np.testing.assert_allclose(yb, ya, rtol=0, atol=1e-5 * np.sqrt(np.mean(ya ** 2)))
    _assert_lowp(ya, M.run_causal(nodes, p, x, seed=3)[:, 0], "served audio -> audio, BF16")
    assert server.stats()["max_batch"] >= 2
    server.close()
    model.close()
