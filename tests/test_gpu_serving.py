"""Serving form: continuous batching through the library's scheduler.

A stream's output must not depend on which other streams share its batches
(the mix changes as streams arrive and leave), requests shorter than a model
step are served from the stream's output FIFO, and streams are admitted by
arena slots."""
import time

import numpy as np
import pytest

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


_COMPLETED = {}


def _drain(server, tags_wanted, timeout=30.0):
    """Waits until every wanted tag has completed (other streams' completions
    are recorded too).  The output buffers of a request must stay alive until
    its tag is reported: the scheduler thread writes them."""
    t0 = time.time()
    while not all(t in _COMPLETED for t in tags_wanted):
        tags, sub, fin = server.poll()
        for t, a, b in zip(tags, sub, fin):
            _COMPLETED[int(t)] = (int(a), int(b))
        if time.time() - t0 > timeout:
            missing = [t for t in tags_wanted if t not in _COMPLETED]
            raise TimeoutError(f"{len(missing)} of {len(tags_wanted)} requests not completed")
        time.sleep(0.001)
    return {t: _COMPLETED[t] for t in tags_wanted}


def _serve(server, stream, z, buffers, tag0, extra=None):
    """Submit one stream's requests (buffer sizes in samples), 2048-sample
    latent frames attached as soon as they are due; returns the output."""
    outs, tags = [], []
    sent, asked = 0, 0
    for i, b in enumerate(buffers):
        asked += b
        need = -(-asked // 2048)
        frames = np.ascontiguousarray(z[sent:need], dtype=np.float32)
        out = np.zeros((b, 1), np.float32)
        outs.append(out)
        tags.append(tag0 + i)
        server.submit([stream], [frames if need > sent else None], [need - sent], [out], [b], [tag0 + i])
        sent = need
        if extra:
            extra(i)
    _drain(server, tags)
    return np.concatenate(outs)[:, 0], frames


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_stream_alone_equals_stream_in_the_mix(cclib, cuda, dtype):
    dec, p = _decoder(2)
    steps = 6
    z = W.signal(3, steps, 128)
    model = api.Model(dec, p, dtype=dtype, max_streams=12, max_steps_per_call=1)
    server = api.Server(model, max_batch=10, bucket=4)
    alone = model.stream(seed=5)
    base = 1_000_000 * (1 if dtype == "bf16" else 2)
    y_alone, _ = _serve(server, alone, z, [2048] * steps, base)
    server.remove(alone)

    # the same stream again, now sharing batches with others that join,
    # submit uneven buffers and leave at different times
    mixed = model.stream(seed=5)
    others = [model.stream(seed=100 + k) for k in range(6)]
    rng = np.random.default_rng(0)
    keep = []

    def traffic(i):
        for k, s in enumerate(others):
            if k <= i + 1:
                b = int(rng.choice([512, 1024, 2048, 4096]))
                frames = rng.standard_normal((max(1, b // 2048), 128)).astype(np.float32)
                out = np.zeros((b, 1), np.float32)
                keep.append((frames, out))
                server.submit([s], [frames], [frames.shape[0]], [out], [b], [base + 10_000 + 100 * k + i])
    y_mixed, _ = _serve(server, mixed, z, [2048] * steps, base + 1000, extra=traffic)
    # same result within the FP32 bar: FP32 layers may pick other reduction
    # shapes for other batch widths
    np.testing.assert_allclose(y_mixed, y_alone, rtol=0, atol=1e-5 * np.sqrt(np.mean(y_alone ** 2)))
    # and both are the reconfigured model's output
    ref = M.run_causal(dec, p, z, seed=5)[:, 0]
    err = np.max(np.abs(y_alone - ref))
    assert err <= (2e-2 * np.abs(ref).max() if dtype == "bf16" else 1e-5 * np.sqrt(np.mean(ref ** 2)))
    stats = server.stats()
    assert stats["max_batch"] >= 2 and stats["stream_steps"] >= 2 * steps
    server.close()


def test_small_buffers_served_from_fifo(cclib, cuda):
    dec, p = _decoder(3)
    z = W.signal(4, 4, 128)
    model = api.Model(dec, p, dtype="bf16", max_streams=4, max_steps_per_call=1)
    server = api.Server(model, max_batch=2, bucket=1)
    a, b = model.stream(seed=9), model.stream(seed=9)
    ya, _ = _serve(server, a, z, [2048] * 4, 3_000_000)
    yb, _ = _serve(server, b, z, [512, 1024, 512, 4096, 1024, 1024], 3_000_100)
    np.testing.assert_allclose(yb, ya, rtol=0, atol=1e-5 * np.sqrt(np.mean(ya ** 2)))
    server.close()


def test_admission_by_arena_slots(cclib, cuda):
    dec, p = _decoder(4)
    model = api.Model(dec, p, dtype="bf16", max_streams=3, max_steps_per_call=1)
    server = api.Server(model, max_batch=2, bucket=1)  # takes one slot for padding
    s1, s2 = model.stream(), model.stream()
    with pytest.raises(api.CCError) as e:
        model.stream()
    assert e.value.status == -4
    server.remove(s1)
    s1.close()
    s3 = model.stream()  # admitted once a slot is free
    z = W.signal(5, 1, 128).astype(np.float32)
    out = np.zeros((2048, 1), np.float32)
    server.submit([s3], [z], [1], [out], [2048], [4_000_007])
    done = _drain(server, [4_000_007])
    assert done[4_000_007][1] >= done[4_000_007][0]
    server.close()


def test_prepare_sets_every_bucket_up_front(cclib, cuda):
    """cc_server_prepare tunes and captures each bucket before serving: the
    later batches need no set-up, every request reports the start of the GPU
    step that completed it (submit <= step start <= done), and the outputs are
    those of an unprepared server."""
    dec, p = _decoder(5)
    z = W.signal(6, 3, 128)
    outs = {}
    for prepared in (False, True):
        model = api.Model(dec, p, dtype="bf16", max_streams=10, max_steps_per_call=1)
        server = api.Server(model, max_batch=8, bucket=4)
        if prepared:
            server.prepare(8)
            st = server.stats()
            assert st["setups"] == 2 and st["batches"] == 0 and st["setup_ns"] > 0  # buckets of 4 and 8
        streams = [model.stream(seed=20 + k) for k in range(6)]
        ys = [[] for _ in streams]
        for t in range(3):
            frames = np.ascontiguousarray(z[t:t + 1], dtype=np.float32)
            bufs = [np.zeros((2048, 1), np.float32) for _ in streams]
            tags = [7_000_000 + 1000 * prepared + 10 * t + k for k in range(len(streams))]
            server.submit(streams, [frames] * len(streams), [1] * len(streams), bufs, [2048] * len(streams), tags)
            got = {}
            t0 = time.time()
            while len(got) < len(tags) and time.time() - t0 < 30:
                tg, sub, step, fin = server.poll(detail=True)
                for a, b, c, d in zip(tg, sub, step, fin):
                    got[int(a)] = (int(b), int(c), int(d))
                time.sleep(0.001)
            assert len(got) == len(tags)
            for tag in tags:
                sub, step, fin = got[tag]
                assert sub <= step <= fin
            for k, b in enumerate(bufs):
                ys[k].append(b[:, 0].copy())
        st = server.stats()
        if prepared:
            assert st["setups"] == 2  # nothing set up while serving
        else:
            assert st["setups"] >= 1
        outs[prepared] = [np.concatenate(y) for y in ys]
        server.close()
        model.close()
    # the autotuner may pick other tile shapes for the same bucket (timing):
    # same result within the FP32 bar
    for a, b in zip(outs[False], outs[True]):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-5 * np.sqrt(np.mean(a ** 2)))
