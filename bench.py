"""Throughput of streamed RAVE-like decoding on GB300 (real-time 48 kHz streams).

One step = one 2048-sample buffer (one latent frame) for every stream of the
batch, through the whole reconfigured decoder: cached convolutions, polyphase
transposed convolutions, aligned residual adds, heads and inverse PQMF.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the FP64 oracle on the host cores)

Prints one JSON line.  ``value`` = output samples per second / 48000 over all
ranks (each rank runs an independent replica: streams are independent).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SR = 48000
METRIC = "real-time 48kHz streams per GB300 (BF16 vs FP32 cached conv); p99 buffer latency"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
SM_COUNT = 152
FP32_LANES_PER_SM = 128

# Concurrent launch chains per step (default): one per 256 streams in the
# low-precision modes (measured best at 256, 1024 and 2048 streams), one in FP32.
def default_sub_batches(dtype, streams):
    return 1 if dtype == "f32" else max(1, streams // 256)

# DRAM bytes (read + write) per tensor-core launch from one ncu capture of a
# step of the workload, keyed by workload, with the SHA-256 prefix of the
# tensor-core kernel source the capture ran: the figure is reported only while
# the source is unchanged (null otherwise, and for other workloads).  The
# decoder's: 152.4 MB read and ~0 written (L2 absorbs the writes within the
# capture) over the 21 tensor-core launches of the fifth step of
# `bench.py --steps 3 --warmup 3 --only-timed` (ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum -k regex:k_conv_tc -s 84 -c 21).
TC_TRAFFIC_PER_LAUNCH = {"decoder-bf16-b256": (7.26e6, "c7836a56a72605f8")}
TC_SOURCE = os.path.join(ROOT, "paper_2204_07064_gb300", "csrc", "cc_kernels_tc.cu")


def tc_source_sha16():
    import hashlib

    with open(TC_SOURCE, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(workload):
    entry = TC_TRAFFIC_PER_LAUNCH.get(workload)
    if entry is None or entry[1] != tc_source_sha16():
        return None
    return entry[0]

WORKLOADS = {
    # name: (dtype, streams, model steps (2048 output samples each) per buffer, model)
    "decoder-bf16-b256": ("bf16", 256, 1, "decoder"),
    "decoder-f16-b256": ("f16", 256, 1, "decoder"),
    "decoder-fp32-b256": ("f32", 256, 1, "decoder"),
    "decoder-fp32-b1": ("f32", 1, 1, "decoder"),
    "decoder-bf16-b1024": ("bf16", 1024, 1, "decoder"),
    "decoder-bf16-b2048": ("bf16", 2048, 1, "decoder"),
    # audio -> audio: the encoder feeding the decoder as one streamed model
    "autoencoder-bf16-b256": ("bf16", 256, 1, "autoencoder"),
    "autoencoder-fp32-b256": ("f32", 256, 1, "autoencoder"),
}
MODEL_NAMES = {"decoder": "RAVE-like decoder, random init",
               "autoencoder": "RAVE-like encoder -> decoder (audio -> audio), random init"}
DEFAULT_WORKLOAD = "decoder-bf16-b256"


def max_over_ranks(ms, dist, device):
    """The slowest rank's time; every rank gets it (replicas: the job ends
    when the last rank ends).  `dist` None means one process."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_streams(streams_per_rank, world, steps, samples_per_step, ms):
    """Real-time 48 kHz streams of the whole job: output samples of every
    rank's streams over `steps` steps, divided by the slowest rank's time."""
    return streams_per_rank * world * samples_per_step * steps / (ms / 1000.0) / SR


def device_free_bytes(dev):
    try:
        import torch

        torch.cuda.synchronize(dev)
        return int(torch.cuda.mem_get_info(dev)[0])
    except Exception:
        return None


def model_memory(model, streams, free_before, free_after):
    """Memory of streaming (section 4.1 reports the cached padding as a constant
    extra 180 kiB per stream): the persistent cache state per stream, the arena
    slot per stream (state plus per-call rows and low-precision mirrors), the
    arena, and the device memory the model took (free-memory delta around its
    creation: weights, arena, bookkeeping)."""
    state, slot = model.state_bytes
    out = {"state_bytes_per_stream": int(state), "slot_bytes_per_stream": int(slot),
           "arena_bytes": int(slot) * int(streams), "device_bytes_model": None}
    if free_before is not None and free_after is not None:
        out["device_bytes_model"] = int(free_before - free_after)
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK, sm_max_mhz=2070.0), "fallback"


def node_bytes(node, u_in, u_out):
    """Algorithmic HBM bytes of one FP32 node for one stream-step: every input
    frame read once and every output frame written once, 4 bytes per value
    (merges read each of their inputs)."""
    op = node["op"]
    if op in ("conv", "convt", "input"):
        return 4 * (u_in * node["c_in"] + u_out * node["c_out"])
    if op == "heads":
        return 4 * u_out * node["c_out"] * 4  # three branches in, one out
    if op == "add":
        return 4 * u_out * node["c_out"] * 3
    return 0


def node_flops(node, frames_out_per_step):
    """Algorithmic FLOPs (2 per MAC) of one node for one stream-step."""
    op = node["op"]
    if op == "conv":
        return 2 * node["c_out"] * node["c_in"] * node["k"] * frames_out_per_step
    if op == "convt":
        return 2 * node["c_in"] * node["c_out"] * node["k"] * frames_out_per_step // node["stride"]
    return 0


def build_decoder(dtype, streams, seed=1, kind="decoder"):
    """The decoder (latent in, audio out) or, for kind "autoencoder", the
    encoder feeding the decoder (audio in, audio out), random weights."""
    from paper_2204_07064_gb300 import api
    from paper_2204_07064_gb300 import workloads as W

    nodes = W.rave_decoder() if kind == "decoder" else W.chain(W.rave_encoder(), W.rave_decoder())
    params = W.init_params(nodes, seed)
    analysis, synthesis = api.pqmf_layer_weights(16, 64, 5.0)
    for i, nd in enumerate(nodes):
        if nd["name"] == "ipqmf":
            params[i] = (synthesis, None)
        if nd["name"] == "pqmf":
            params[i] = (analysis, None)
    model = api.Model(nodes, params, dtype=dtype, max_streams=streams, max_steps_per_call=1)
    return nodes, params, model


def autoencoder(dtype, streams, seed=4, steps_per_call=1):
    """The encoder feeding the decoder (audio -> audio), random weights, the
    16-band PQMF pair; a low-precision model is built without fused residual
    units (the backward needs each convolution's output)."""
    from paper_2204_07064_gb300 import api
    from paper_2204_07064_gb300 import workloads as W

    nodes = W.chain(W.rave_encoder(), W.rave_decoder())
    params = W.init_params(nodes, seed)
    analysis, synthesis = api.pqmf_layer_weights(16, 64, 5.0)
    for i, nd in enumerate(nodes):
        if nd["name"] == "pqmf":
            params[i] = (analysis, None)
        if nd["name"] == "ipqmf":
            params[i] = (synthesis, None)
    model = api.Model(nodes, params, dtype=dtype, max_streams=streams, max_steps_per_call=steps_per_call,
                      fuse_units=dtype == "f32")
    return nodes, params, model


def run_differentiate(args):
    """Differentiation form: the encoder + decoder (audio -> audio) with a BF16
    forward on the tensor cores (--diff-dtype f32: FFMA) and FP32 gradients,
    --diff-streams streams of --diff-chunks 2048-sample chunks of N(0, 0.1^2)
    audio (60 s at 48 kHz = 1407 chunks), streamed through torch.autograd with
    one compact state checkpoint per chunk, then the chunked backward (loss =
    sum(r * y), r ~ N(0, 1) seeded; gradients of every weight and bias and of
    the input audio).  The forward and the backward are timed with CUDA
    events; audio seconds differentiated per second = streams x chunks x 2048
    / 48000 / (forward + backward seconds).  A second, shorter pass with every
    backward kernel bracketed by events gives the kernels' shares, the nodes
    that cost most, and the roofline of the dominant class (FP32 FFMA:
    ALU-bound)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2204_07064_gb300 import api
    from paper_2204_07064_gb300 import autograd as AG

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    dtype = args.diff_dtype
    count, chunks, cs = args.diff_streams, args.diff_chunks, args.diff_chunk_steps
    if chunks % cs:
        raise SystemExit("--diff-chunks must be a multiple of --diff-chunk-steps")
    nodes, params, model = autoencoder(dtype, count, steps_per_call=cs)
    streams = [model.stream(seed=1000 + s) for s in range(count)]
    runner = AG.StreamedRunner(model, params, streams, cs)
    n = chunks * 2048
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.standard_normal((count, n, 1)) * 0.1, dtype=torch.float32, device=dev)
    r = torch.tensor(rng.standard_normal((count, n, 1)), dtype=torch.float32, device=dev)
    free0 = device_free_bytes(dev)

    def one_pass(xx, rr, events=None):
        xx = xx.detach().requires_grad_(True)
        runner.grads.zero()
        for s in streams:
            s.reset()
        if events:
            events[0].record()
        y = AG.streamed(xx, runner)
        if events:
            events[1].record()
        (y * rr).sum().backward()
        if events:
            events[2].record()
        return xx.grad

    warm = min(chunks, 8 * cs)
    for _ in range(max(1, args.warmup // 3)):
        one_pass(x[:, :warm * 2048], r[:, :warm * 2048])
    torch.cuda.synchronize()
    model.device_status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    t0 = time.time()
    gx = one_pass(x, r, ev)
    torch.cuda.synchronize()
    t1 = time.time()
    clk = clocks.stop(window=(t0, t1))
    model.device_status()
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    free1 = device_free_bytes(dev)
    assert torch.isfinite(gx).all()
    audio_s = count * n / SR
    snap = api.snapshot_bytes(model)
    slot = model.state_bytes[1]

    # kernel classes of the backward over a window of chunks (events around
    # every launch; the absolute times include that overhead, the shares are
    # what the roofline uses)
    win = min(chunks, 32 * cs)
    runner.grads.timing(True)
    one_pass(x[:, :win * 2048], r[:, :win * 2048])
    torch.cuda.synchronize()
    classes = runner.grads.timing_read()
    per_node = runner.grads.timing_read_nodes()
    runner.grads.timing(False)
    ev_total = sum(v[0] for v in classes.values())
    info_u = [model.node_info(i)["frames_per_step"] for i in range(len(nodes))]
    conv_flops = sum(node_flops(nd, info_u[i]) for i, nd in enumerate(nodes) if nd["op"] in ("conv", "convt"))
    # dL/dW and dL/dx each cost the forward's multiply-adds: per stream-step
    per_class_flops = {"weight": conv_flops, "data": conv_flops}
    pk, pk_kind = peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    kernels = {}
    for c, (ms, cnt) in classes.items():
        e = {"launches": cnt, "event_ms": ms, "share": ms / ev_total if ev_total else None}
        if c in per_class_flops and cnt:
            # the class's share of the event pass, applied to the timed backward
            e["achieved_tflops"] = per_class_flops[c] * count * chunks / (bwd_ms / 1000.0 * e["share"]) / 1e12
        kernels[c] = e
    top = []
    for i, c, ms, cnt in sorted(per_node, key=lambda e: -e[2])[:10]:
        e = {"node": nodes[i]["name"] or nodes[i]["op"], "class": c, "us_per_chunk": 1000.0 * ms / win,
             "share": ms / ev_total if ev_total else None}
        if c in ("weight", "data"):
            e["event_tflops"] = node_flops(nodes[i], info_u[i]) * count * win / (ms / 1000.0) / 1e12
        top.append(e)
    dom = max(("weight", "data"), key=lambda c: classes[c][0])
    achieved = kernels[dom]["achieved_tflops"]
    line = {
        "metric": "streamed forward + backward, audio seconds differentiated per second",
        "value": audio_s / ((fwd_ms + bwd_ms) / 1000.0),
        "unit": "audio s / s", "higher_is_better": True, "dtype": f"{dtype} forward, f32 gradients",
        "data": "synthetic", "n_gpus": 1,
        "ms": {"forward_with_checkpoints": fwd_ms, "backward": bwd_ms},
        "config": {"workload": f"autoencoder-{dtype}-diff-{count}x{chunks}", "streams": count, "chunks": chunks,
                   "chunk_samples": 2048 * cs, "audio_seconds_per_stream": n / SR,
                   "loss": "sum(r * y), r ~ N(0,1) seeded", "input": "N(0, 0.1^2) audio, seed 4",
                   "gradients": "every weight and bias, and the input audio"},
        "checkpoints": {"bytes_per_stream_per_chunk": snap, "arena_slot_bytes": slot,
                        "total_bytes": (chunks // cs + 1) * count * snap},
        "device_memory_used_bytes": free0 - free1 if free0 and free1 else None,
        "backward_kernels": {"window_chunks": win, "classes": kernels, "top_nodes": top,
                             "note": "event-bracketed pass over the first window_chunks chunks; shares of its "
                                     "summed event times"},
        "roofline": {"bound": "alu", "kernel": f"k_bwd_{dom} (FP32 FFMA, 64x64 tiles)", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "achieved_from": "the class's algorithmic FLOPs over the whole pass / (timed backward x its "
                                      "share of the event pass)",
                     "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"},
        "clocks": clk,
    }
    print(json.dumps(line))
    model.close()


def throughput_at(batch, steps=200, warmup=3):
    """Real-time streams at `batch` streams (BF16 decoder, one 2048-sample
    buffer per step), the step captured as a CUDA graph of one launch chain
    per 256 streams, timed with CUDA events over `steps` steps."""
    import torch

    from paper_2204_07064_gb300 import workloads as W

    _, _, model = build_decoder("bf16", batch)
    ss = [model.stream(seed=s) for s in W.stream_seeds(77, batch)]
    dev = torch.device("cuda", torch.cuda.current_device())
    z = torch.randn((warmup + steps, batch, 1, 128), device=dev)
    x_in = torch.empty_like(z[0])
    y = torch.empty((batch, 2048, 1), device=dev)
    nsub = default_sub_batches("bf16", batch)
    bounds = [round(k * batch / nsub) for k in range(nsub + 1)]
    side = [torch.cuda.Stream() for _ in range(nsub)]

    def launch(main):
        fork = torch.cuda.Event()
        fork.record(main)
        for k in range(nsub):
            side[k].wait_event(fork)
            model.process_batch(ss[bounds[k]:bounds[k + 1]], x_in[bounds[k]:bounds[k + 1]],
                                y[bounds[k]:bounds[k + 1]], cuda_stream=side[k])
        for k in range(nsub):
            main.wait_stream(side[k])

    st = torch.cuda.current_stream()
    for i in range(warmup):
        x_in.copy_(z[i])
        launch(st)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(st)
    with torch.cuda.graph(graph, stream=cap, capture_error_mode="relaxed"):
        launch(cap)
    st.wait_stream(cap)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(steps):
        x_in.copy_(z[warmup + i])
        graph.replay()
    e1.record(st)
    torch.cuda.synchronize()
    model.device_status()
    ms = e0.elapsed_time(e1) / steps
    del graph
    model.close()
    return batch * 2048 / (ms / 1000.0) / SR, ms


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms.  Each row is
    time-stamped by nvidia-smi; `stop(window)` keeps the rows that fall inside
    the given wall-clock window (the timed region)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    @staticmethod
    def parse(out, window=None, fallback=None):
        """Summary of nvidia-smi rows; with `window` = (t0, t1) in time.time()
        seconds, only the rows stamped inside it.  When no row falls inside
        (a timed region shorter than the sampling interval), the rows inside
        `fallback` (a wall-clock interval of the same load right after it)
        are used instead, and the summary says so."""
        import datetime
        rows = []
        for line in out.strip().splitlines():
            r = [f.strip() for f in line.split(",")]
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(r[2]), float(r[3]),
                             {name for name, v in zip(ClockSampler.REASONS, r[6:10]) if v.lower() == "active"}))
            except (ValueError, IndexError):
                continue
        if not rows:
            return None

        def inside(iv):
            return [x for x in rows if iv is None or iv[0] <= x[0] <= iv[1]]

        picked, note = inside(window), None
        if not picked and window is not None and fallback is not None:
            picked = inside(fallback)
            note = "no sample inside the timed region (shorter than the sampling interval); samples from 0.3 s " \
                   "of replays of the same step right after it"
        if not picked:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "samples_total": len(rows),
                    "note": "no sample fell inside the timed region"}
        out = {"sm_mhz": statistics.median(x[1] for x in picked), "sm_max_mhz": max(x[2] for x in picked),
               "reasons": sorted(set().union(*(x[3] for x in picked))), "samples": len(picked),
               "samples_total": len(rows)}
        if note:
            out["note"] = note
        return out

    def stop(self, window=None, fallback=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out, window, fallback)


def oracle_sample(steps, seed=1, stream_seed=11, warmup=1, kind="decoder", threads=1):
    """FP64 oracle streaming of the same model (decoder, or encoder -> decoder),
    one stream: `warmup` untimed buffers, then `steps` timed buffers of one
    model step each (one wall time each).  Runs in a subprocess with `threads`
    BLAS threads; returns audio seconds / wall."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import model as M, pqmf
from paper_2204_07064_gb300 import workloads as W
if {kind!r} == "decoder":
    nodes = W.rave_decoder()
    z = W.signal(5, {warmup} + {steps}, 128)
    n = 1
else:
    nodes = W.chain(W.rave_encoder(), W.rave_decoder())
    z = W.signal(5, ({warmup} + {steps}) * 2048, 1, std=0.1)
    n = 2048
p = W.init_params(nodes, {seed})
_, g, _, _ = pqmf.design(16, 64)
for i, nd in enumerate(nodes):
    if nd["name"] == "ipqmf":
        p[i] = (pqmf.synthesis_weights(g), None)
    if nd["name"] == "pqmf":
        p[i] = (pqmf.analysis_weights(g), None)
s = M.Stream(nodes, p, seed={stream_seed})
for i in range({warmup}):
    s.process(z[i * n:(i + 1) * n])
walls = []
for i in range({warmup}, {warmup} + {steps}):
    t = time.perf_counter()
    s.process(z[i * n:(i + 1) * n])
    walls.append(time.perf_counter() - t)
print(json.dumps({{"wall": sum(walls), "walls": walls, "audio_s": {steps} * 2048 / {SR}}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=max(600.0, 0.5 * (steps + warmup)))
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["audio_s"] / d["wall"], d


def run_reference(args):
    """The oracle as the reference arm: FP64 NumPy streaming on host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dtype, streams, frames, kind = WORKLOADS[args.workload]
    # one process; each step is one 2048-sample buffer of one stream
    value, d = oracle_sample(args.steps, warmup=args.warmup, kind=kind)
    walls = d["walls"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "streams",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(walls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "streams": streams, "buffer_samples": 2048 * frames,
                   "note": "oracle timed on 1 stream x 1 buffer per step (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "streams", "cores": 1, "kind": "oracle",
                         "sample": f"1 stream x 1 buffer of 2048 samples per step, {args.steps} steps, "
                                   f"FP64 NumPy, 1 BLAS thread ({d['wall']:.1f} s)"},
        "e2e": {"value": value, "unit": "streams", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def serve_once(args, kind, cap, fixed, run_s, warm_s, prepare=True):
    """One serving run through the library's scheduler (cc_server_*), BF16.
    kind "decoder": latent frames in, audio out; streams arrive Poisson(200/s),
    live U[5, 60] s and draw a buffer size from {512, 1024, 2048, 4096}.
    kind "autoencoder": the encoder feeding the decoder, 2048-sample audio
    buffers in and out.  fixed > 0: that many streams of 2048-sample buffers
    for the whole run instead of arrivals.  Each stream submits one request
    per buffer period, paced in wall-clock time, at most 4 in flight.
    Latency = submit -> output ready; deadline = the buffer's duration."""
    from paper_2204_07064_gb300 import api

    if kind == "decoder":
        nodes, params, model = build_decoder("bf16", cap + 1)
    else:
        nodes, params, model = build_decoder("bf16", cap + 1, kind="autoencoder")
    io = model.io
    cin = io["in_channels"]
    bucket = max(32, -(-cap // 64))
    server = api.Server(model, max_batch=cap, bucket=bucket, use_graphs=True, autotune=True)
    t_prep = time.perf_counter()
    if prepare:
        server.prepare(cap)
    t_prep = time.perf_counter() - t_prep
    rng = np.random.default_rng(3)
    lam = 200.0
    sizes = np.array([512, 1024, 2048, 4096]) if (kind == "decoder" and not fixed) else np.array([2048])
    bmax = int(sizes.max())
    ring = 4  # output buffers per stream (requests in flight per stream)
    pool_frames = 4096
    pool = rng.standard_normal((pool_frames * (2048 if kind != "decoder" else 1), cin)).astype(np.float32)
    if kind != "decoder":
        pool *= 0.1
    outs = np.zeros((cap, ring, bmax), np.float32)
    pool_base, out_base = pool.ctypes.data, outs.ctypes.data
    active = np.zeros(cap, bool)
    handles = [None] * cap
    hptr = np.zeros(cap, np.uint64)
    B = np.zeros(cap, np.int64)
    next_due = np.zeros(cap, np.int64)
    end_ns = np.zeros(cap, np.int64)
    asked = np.zeros(cap, np.int64)
    sent = np.zeros(cap, np.int64)
    nreq = np.zeros(cap, np.int64)
    outstanding = np.zeros(cap, np.int64)
    gen = np.zeros(cap, np.int64)
    t_start = time.perf_counter_ns()
    t_meas = t_start + int(warm_s * 1e9)
    t_end = t_meas + int(run_s * 1e9)
    # results in preallocated arrays (the client must keep up with ~0.5 M
    # requests/s at 24 k streams: no per-request Python objects, no GC pauses)
    expect = int((run_s + 2.0) * cap * SR / int(sizes.min()) * 1.2) + 1024
    res = np.zeros((4, expect), np.float32)  # latency, wait, step (ms), buffer size
    nres = 0
    import gc
    gc_was = gc.isenabled()
    gc.disable()
    rejected = admitted = 0
    delivered = 0
    conc = []
    clocks = ClockSampler(0)
    sampled = False
    wall_meas = None
    st0 = None
    last = t_start
    if fixed:
        for i in range(cap):
            handles[i] = model.stream(seed=i)
            hptr[i] = handles[i].handle.value
            active[i], B[i], end_ns[i] = True, 2048, 1 << 62
            next_due[i] = t_start + int(rng.uniform(0, 2048 / SR) * 1e9)
    while True:
        now = time.perf_counter_ns()
        if now >= t_end:
            break
        if not sampled and now >= t_meas:
            clocks.start()
            sampled = True
            wall_meas = time.time()
            st0 = server.stats()
        dt = (now - last) / 1e9
        last = now
        if not fixed:
            # departures (once nothing is in flight), then Poisson arrivals
            gone = np.nonzero(active & (end_ns <= now) & (outstanding == 0))[0]
            for i in gone:
                server.remove(handles[i])
                handles[i].close()
                handles[i] = None
                active[i] = False
            for _ in range(rng.poisson(lam * dt)):
                free = np.nonzero(~active)[0]
                if len(free) == 0:
                    rejected += 1
                    continue
                i = int(free[0])
                try:
                    handles[i] = model.stream(seed=int(rng.integers(1 << 62)))
                except api.CCError:
                    rejected += 1
                    continue
                admitted += 1
                hptr[i] = handles[i].handle.value
                active[i], B[i] = True, int(rng.choice(sizes))
                next_due[i] = now
                end_ns[i] = now + int(rng.uniform(5, 60) * 1e9)
                asked[i] = sent[i] = nreq[i] = outstanding[i] = 0
                gen[i] += 1
        due = np.nonzero(active & (next_due <= now) & (outstanding < ring))[0]
        if len(due):
            b = B[due]
            if kind == "decoder":
                # latent frames as soon as the output they make is asked for
                asked[due] += b
                need = -(-asked[due] // 2048)
                n_in = need - sent[due]
                sent[due] = need
                frame = (due * 61 + nreq[due] * 3) % (pool_frames - 2)
                in_ptr = (pool_base + frame * cin * 4).astype(np.uint64)
            else:
                n_in = b
                frame = (due * 61 + nreq[due] * 3) % (pool_frames - 2)
                in_ptr = (pool_base + frame * 2048 * 4).astype(np.uint64)
            out_ptr = (out_base + ((due * ring + nreq[due] % ring) * bmax) * 4).astype(np.uint64)
            tags = ((gen[due] << 40) | (due << 24) | (nreq[due] & 0xFFFFFF)).astype(np.uint64)
            server.submit_raw(len(due), np.ascontiguousarray(hptr[due]), in_ptr, np.asarray(n_in, np.int64),
                              out_ptr, b.astype(np.int64), tags)
            nreq[due] += 1
            outstanding[due] += 1
            next_due[due] += (b * 1e9 / SR).astype(np.int64)
        tags, sub, step, fin = server.poll(detail=True)
        if len(tags):
            idx = ((tags >> 24) & 0xFFFF).astype(np.int64)
            g = (tags >> 40).astype(np.int64)
            live = g == gen[idx]
            outstanding -= np.bincount(idx[live], minlength=cap)
            if now >= t_meas:
                k = min(len(tags), expect - nres)
                res[0, nres:nres + k] = (fin[:k] - sub[:k]) / 1e6
                res[1, nres:nres + k] = (step[:k] - sub[:k]) / 1e6
                res[2, nres:nres + k] = (fin[:k] - step[:k]) / 1e6
                res[3, nres:nres + k] = B[idx[:k]]
                nres += k
                delivered += int(B[idx].sum())
        if now >= t_meas:
            conc.append(int(active.sum()))
        time.sleep(0.0005)
    clk = clocks.stop((wall_meas, time.time())) if sampled else None
    if gc_was:
        gc.enable()
    st = server.stats()
    server.close()
    model.close()
    lat, wait, stepd, lat_b = res[0, :nres], res[1, :nres], res[2, :nres], res[3, :nres]
    per_b = {}
    for b in sizes:
        m = lat_b == b
        if m.any():
            dl = 1000.0 * b / SR
            miss = m & (lat >= dl)
            e = {"p50_ms": float(np.percentile(lat[m], 50)), "p99_ms": float(np.percentile(lat[m], 99)),
                 "max_ms": float(lat[m].max()), "deadline_ms": dl, "met": float(np.mean(lat[m] < dl)),
                 "requests": int(m.sum())}
            if miss.any():
                # where a missed request's time went: waiting for its step to
                # start (queue, the previous batch, the host) vs the step itself
                e["missed"] = {"count": int(miss.sum()), "wait_p50_ms": float(np.median(wait[miss])),
                               "step_p50_ms": float(np.median(stepd[miss])),
                               "wait_max_ms": float(wait[miss].max()), "step_max_ms": float(stepd[miss].max())}
            per_b[str(int(b))] = e
    meas = {k: st[k] - (st0 or {}).get(k, 0) for k in ("batches", "stream_steps", "gpu_ns", "setups", "setup_ns")}
    return {
        "value": delivered / run_s / SR, "cap": cap, "fixed": fixed,
        "latency_ms": {"p50": float(np.percentile(lat, 50)) if len(lat) else None,
                       "p99": float(np.percentile(lat, 99)) if len(lat) else None,
                       "max": float(lat.max()) if len(lat) else None,
                       "wait_p50": float(np.percentile(wait, 50)) if len(wait) else None,
                       "step_p50": float(np.percentile(stepd, 50)) if len(stepd) else None,
                       "per_buffer": per_b,
                       "met_deadline": float(np.mean([v["met"] for v in per_b.values()])) if per_b else None},
        "streams": {"mean_concurrent": float(np.mean(conc)) if conc else 0, "max_concurrent": int(max(conc or [0])),
                    "admitted": admitted, "rejected": rejected},
        "server": {"bucket": bucket, "prepare_s": t_prep if prepare else None,
                   "batches": meas["batches"], "stream_steps": meas["stream_steps"],
                   "mean_batch": meas["stream_steps"] / max(1, meas["batches"]), "max_batch": st["max_batch"],
                   "gpu_busy": meas["gpu_ns"] / (run_s * 1e9), "setups_while_serving": meas["setups"],
                   "setup_ms_while_serving": meas["setup_ns"] / 1e6},
        "clocks": clk,
    }


def run_serving(args):
    """Serving form through the library's scheduler.  Without --serve-sweep:
    one run (Poisson arrivals, or --serve-fixed N streams).  With
    --serve-sweep N1,N2,..: fixed-N runs of 2048-sample buffers at growing N
    (the capacity sweep), stopping after the first N whose p99 latency reaches
    the buffer duration.  Every bucket is tuned and captured before the
    measured region (cc_server_prepare) unless --serve-no-prepare."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    kind = args.serve_model
    prepare = not args.serve_no_prepare
    base = {"metric": METRIC, "unit": "streams", "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic"}
    if args.serve_sweep:
        points = []
        for n in [int(v) for v in args.serve_sweep.split(",")]:
            r = serve_once(args, kind, n, n, args.serve_seconds, args.serve_warmup, prepare)
            points.append(r)
            print(json.dumps({"sweep_point": n, "value": r["value"], "p99_ms": r["latency_ms"]["p99"],
                              "max_ms": r["latency_ms"]["max"], "gpu_busy": r["server"]["gpu_busy"]}),
                  file=sys.stderr, flush=True)
            if r["latency_ms"]["p99"] is None or r["latency_ms"]["p99"] >= 2048 / SR * 1000.0:
                break
        ok = [p for p in points if p["latency_ms"]["p99"] is not None and p["latency_ms"]["p99"] < 2048 / SR * 1000.0]
        line = dict(base, value=max([p["value"] for p in ok], default=0.0),
                    config={"workload": f"serving-sweep-{kind}-bf16", "buffer_samples": 2048,
                            "seconds_per_point": args.serve_seconds, "warmup_s": args.serve_warmup,
                            "prepared": prepare},
                    sweep=points,
                    note="value: the largest N whose p99 stayed under the 42.7 ms buffer")
    else:
        fixed = args.serve_fixed
        cap = fixed if fixed else args.serve_cap
        r = serve_once(args, kind, cap, fixed, args.serve_seconds, args.serve_warmup, prepare)
        line = dict(base, **{k: v for k, v in r.items() if k not in ("cap", "fixed")})
        line["config"] = {"workload": f"serving-{kind}-bf16" + (f"-fixed{cap}" if fixed else ""),
                          "arrivals_per_s": 0 if fixed else 200.0, "cap_streams": cap,
                          "buffer_samples": "2048" if (fixed or kind != "decoder") else "U{512,1024,2048,4096}",
                          "lifetime_s": None if fixed else "U[5,60]", "seconds": args.serve_seconds,
                          "prepared": prepare}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-l2", action="store_true", help="write 256 MB between steps")
    ap.add_argument("--sub-batches", type=int, default=0,
                    help="split each step's streams over this many CUDA streams (0: workload default)")
    ap.add_argument("--no-graph", action="store_true", help="launch each step's chains directly")
    ap.add_argument("--graph", action="store_true",
                    help="replay each step from a CUDA graph even with one chain (input copied into its buffer)")
    ap.add_argument("--only-timed", action="store_true",
                    help="skip the e2e, FP32-comparison and CPU-baseline measurements (profiling)")
    ap.add_argument("--serving", action="store_true", help="run the serving simulation instead")
    ap.add_argument("--serve-seconds", type=float, default=120.0)
    ap.add_argument("--serve-warmup", type=float, default=10.0)
    ap.add_argument("--serve-cap", type=int, default=2048)
    ap.add_argument("--serve-fixed", type=int, default=0, help="N fixed streams of 2048-sample buffers")
    ap.add_argument("--serve-model", default="decoder", choices=["decoder", "autoencoder"])
    ap.add_argument("--serve-sweep", default="", help="comma-separated fixed stream counts (capacity sweep)")
    ap.add_argument("--serve-no-prepare", action="store_true", help="set buckets up lazily while serving")
    ap.add_argument("--differentiate", action="store_true",
                    help="time the streamed forward + hand-written backward of the encoder + decoder")
    ap.add_argument("--diff-streams", type=int, default=32)
    ap.add_argument("--diff-chunks", type=int, default=1407, help="2048-sample chunks per stream (1407 = 60 s)")
    ap.add_argument("--diff-chunk-steps", type=int, default=1, help="model steps per checkpointed chunk")
    ap.add_argument("--diff-dtype", default="bf16", choices=["bf16", "f16", "f32"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.differentiate:
        return run_differentiate(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2204_07064_gb300 import workloads as W

    dtype, streams, frames, kind = WORKLOADS[args.workload]
    free0 = device_free_bytes(dev)
    nodes, params, model = build_decoder(dtype, streams, kind=kind)
    memory = model_memory(model, streams, free0, device_free_bytes(dev))
    seeds = W.stream_seeds(1000 + rank, streams)
    ss = [model.stream(seed=s) for s in seeds]
    rng = np.random.default_rng(rank)
    steps_total = args.warmup + args.steps
    io = model.io
    in_shape = (frames * io["in_per_step"], io["in_channels"])  # one buffer of one stream
    in_std = 1.0 if kind == "decoder" else 0.1  # latents N(0, 1); audio N(0, 0.1^2)
    z = torch.from_numpy(in_std * rng.standard_normal((steps_total, streams) + in_shape,
                                                      dtype=np.float32)).to(dev)
    y = torch.empty((streams, 2048 * frames, 1), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev) if args.flush_l2 else None
    st = torch.cuda.current_stream()

    # one step = every stream advances one buffer; the streams are split into
    # sub-batches launched on separate CUDA streams so that the launch chains
    # overlap (each chain is latency-bound at this batch size)
    nsub = args.sub_batches or default_sub_batches(dtype, streams)
    nsub = max(1, min(nsub, streams))
    bounds = [round(k * streams / nsub) for k in range(nsub + 1)]
    side = [torch.cuda.Stream() for _ in range(nsub)]
    x_in = torch.empty_like(z[0])  # a captured graph's input buffer (filled each step)

    def launch_step(main, x):
        if nsub == 1:
            model.process_batch(ss, x, y, cuda_stream=main)
            return
        fork = torch.cuda.Event()
        fork.record(main)
        for k in range(nsub):
            a, b = bounds[k], bounds[k + 1]
            side[k].wait_event(fork)
            model.process_batch(ss[a:b], x[a:b], y[a:b], cuda_stream=side[k])
        for k in range(nsub):
            main.wait_stream(side[k])

    for i in range(args.warmup):
        launch_step(st, z[i])
    torch.cuda.synchronize()
    model.device_status()
    # One chain: each step's launches go out directly and read that step's
    # input where it lies (the chains of consecutive steps follow each other
    # with programmatic dependent launch).  Several chains: the step (fork,
    # chains, join) is one CUDA graph, fed by copying the input into its
    # buffer.  On one GB300 at 256 streams the two measured 0.245 and 0.251 ms
    # per step; the copy and the graph boundary make the difference.
    graph = None
    if (nsub > 1 and not args.no_graph) or args.graph:
        # the whole step (fork, every sub-batch's launch chain, join) as one
        # CUDA graph; the batch slot lists were uploaded during the warm-up
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(st)
        with torch.cuda.graph(graph, stream=cap, capture_error_mode="relaxed"):
            launch_step(cap, x_in)
        st.wait_stream(cap)
        torch.cuda.synchronize()

    def step(i):
        if graph is not None:
            x_in.copy_(z[i])
            graph.replay()
        else:
            launch_step(st, z[i])

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    model.device_status()

    # timed region: K steps bracketed by per-step events on the launching stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.time()
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()
        starts[k].record(st)
        step(args.warmup + k)
        ends[k].record(st)
    torch.cuda.synchronize()
    wall1 = time.time()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    # a timed region shorter than the clock sampler's reach: the same step is
    # replayed for 0.3 s right after it, at the same load, and the clock
    # samples come from that window (the line's clocks.note says so)
    clock_window = None
    if wall1 - wall0 < 0.25:
        wc0 = time.time()
        while time.time() - wc0 < 0.3:
            for i in range(50):
                step(args.warmup + i % args.steps)
            torch.cuda.synchronize()
        clock_window = (wc0, time.time())
    # the first K2 = min(K, 500) of those steps again with the library's
    # per-launch events (kernel durations for the roofline; kept out of the
    # headline timing); the e2e and FP32 passes below run K2 steps as well
    k2 = min(args.steps, 500)
    model.timing(True)
    for k in range(k2):
        if flush is not None:
            flush.zero_()
        model.process_batch(ss, z[args.warmup + k], y)
    torch.cuda.synchronize()
    clk = clocks.stop((wall0, wall1), fallback=clock_window or (wall1, time.time()))
    node_ms, node_launches = model.timing_read()
    model.timing(False)
    total_ms = max_over_ranks(total_ms, dist, dev)
    samples = streams * 2048 * frames * args.steps * world
    value = whole_job_streams(streams, world, args.steps, 2048 * frames, total_ms)

    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value,
                              "unit": "streams", "ms_per_step": total_ms / args.steps,
                              "config": {"workload": args.workload}, "note": "--only-timed"}))
        return
    # end to end through the C ABI with pinned host buffers (copies in the timed region)
    zh = torch.empty((streams,) + in_shape, dtype=torch.float32).pin_memory()
    zh.copy_(z[0].cpu())
    yh = torch.empty((streams, 2048 * frames, 1), dtype=torch.float32).pin_memory()
    e_starts = [torch.cuda.Event(enable_timing=True) for _ in range(k2)]
    e_ends = [torch.cuda.Event(enable_timing=True) for _ in range(k2)]
    if dist:
        dist.barrier()
    for k in range(k2):
        e_starts[k].record(st)
        model.process_batch(ss, zh, yh)
        e_ends[k].record(st)
        e_ends[k].synchronize()
    e2e_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(e_starts, e_ends)), dist, dev)
    e2e_value = whole_job_streams(streams, world, k2, 2048 * frames, e2e_ms)

    # roofline of the dominant kernel class: the contractions on the tensor
    # cores (FFMA in FP32 mode).  Their algorithmic FLOPs per step divided by
    # their share of the timed step; the share comes from the per-launch
    # event pass, whose absolute times break the launch overlap and so are
    # not used as durations
    info_u = [model.node_info(i)["frames_per_step"] for i in range(len(nodes))]

    def on_tensor_cores(nd):
        return dtype != "f32" and nd["op"] in ("conv", "convt") and nd["c_in"] % 64 == 0 and nd["c_out"] % 8 == 0

    main_nodes = [i for i, n in enumerate(nodes)
                  if (on_tensor_cores(n) if dtype != "f32" else n["op"] in ("conv", "convt"))]
    flops = sum(node_flops(nodes[i], info_u[i]) for i in main_nodes) * streams * frames
    ev_total = sum(node_ms)
    main_ms = sum(node_ms[i] for i in main_nodes)
    main_launches = sum(node_launches[i] for i in main_nodes)
    share = main_ms / ev_total if ev_total > 0 else 1.0
    step_ms_mean = total_ms / args.steps
    pk, pk_kind = peaks()
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = flops / (step_ms_mean * share / 1000.0) / 1e12
    timing_note = ("algorithmic FLOPs per step / (timed ms per step x the class's share of the per-launch "
                   "event pass)")
    if dtype == "f32":
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "kernel": "cached conv / polyphase convT contractions (FFMA)",
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {pk.get('sm_max_mhz', 2070.0):.0f} MHz"}
    else:
        peak = pk.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic(args.workload),
                "kernel": "tcgen05 implicit-GEMM contractions (k_conv_tc)",
                "peak_source": f"bf16 burst, {pk_kind}"}
    roof.update({"achieved_from": timing_note, "share_of_step": share,
                 "launches_per_step": main_launches / k2 if k2 else None,
                 "event_pass_avg_launch_us": 1000.0 * main_ms / main_launches if main_launches else None,
                 "tc_source_sha16": tc_source_sha16()})
    # every other kernel of the step: algorithmic HBM bytes per launch over its
    # average launch time in the event pass (a lower bound on its rate: events
    # around a launch add their own latency)
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    kernels = []
    for i, nd in enumerate(nodes):
        if node_launches[i] == 0 or i in main_nodes:
            continue
        u_in = info_u[nd["inputs"][0]] if nd["inputs"] else info_u[i]
        b = node_bytes(nd, u_in, info_u[i]) * streams * frames
        avg_s = node_ms[i] / node_launches[i] / 1000.0
        kname = {"input": "k_input", "heads": "k_heads", "add": "k_add"}.get(nd["op"], "FP32 conv kernel")
        kernels.append({"node": nd["name"] or nd["op"], "kernel": kname, "bound": "hbm",
                        "bytes_per_launch": b, "avg_launch_us": avg_s * 1e6,
                        "achieved_gbs": b / avg_s / 1e9, "peak_gbs": hbm_peak,
                        "frac": b / avg_s / 1e9 / hbm_peak, "share_of_step": node_ms[i] / ev_total if ev_total else None})
    roof_others = {"peak_source": f"hbm copy, {pk_kind}", "kernels": kernels,
                   "note": "k_advance (16 bytes per stream) is not timed per launch"}

    model.device_status()  # raises if a bounded device wait gave up

    # the same batch through the FP32 (FFMA) path: the metric compares both
    fp32_cmp = None
    if dtype != "f32":
        model32 = build_decoder("f32", streams, kind=kind)[2]
        ss32 = [model32.stream(seed=s) for s in seeds]
        for i in range(args.warmup):
            model32.process_batch(ss32, z[i], y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for k in range(k2):
            model32.process_batch(ss32, z[args.warmup + k], y)
        e1.record(st)
        torch.cuda.synchronize()
        ms32 = max_over_ranks(e0.elapsed_time(e1) / k2, dist, dev)
        fp32_cmp = {"value": whole_job_streams(streams, world, 1, 2048 * frames, ms32), "unit": "streams",
                    "ms_per_step": ms32, "dtype": "f32", "speedup_lowp_over_fp32": (ms32 / (total_ms / args.steps))}
        model32.close()

    # the same decoder at larger batches (one chain per 256 streams): where the
    # step stops being latency-bound
    by_batch = None
    if dtype != "f32" and streams == 256 and world == 1 and kind == "decoder":
        by_batch = {}
        fl = sum(node_flops(nodes[i], info_u[i]) for i in main_nodes)  # per stream-step, tensor-core layers
        for b in (1024, 2048):
            v, ms_b = throughput_at(b)
            tf = v * SR / 2048 * fl / 1e12
            by_batch[str(b)] = {"value": v, "unit": "streams", "ms_per_step": ms_b,
                                "achieved_tflops": tf, "frac_of_bf16_peak": tf / pk.get("bf16_tflops", 1900.0)}

    step_sorted = sorted(step_ms)
    p50 = float(np.percentile(step_ms, 50))
    p99 = float(np.percentile(step_ms, 99))
    launches_per_step = model.chain_launches * nsub  # every launch of one step's chains
    line = {
        "metric": METRIC, "value": value, "unit": "streams", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": args.workload, "model": MODEL_NAMES[kind],
                   "streams_per_gpu": streams, "buffer_samples": 2048 * frames, "sample_rate": SR,
                   "concurrent_chains": nsub, "cuda_graph": graph is not None,
                   "input": ("copied into the captured graph's input buffer" if graph is not None
                             else "read in place from the step's resident batch"),
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps" if flush is not None else
                   "working set per step > L2 (arena + weights)",
                   "samples_per_s": samples / (total_ms / 1000.0)},
        "throughput_by_batch": by_batch,
        "latency_ms": {"p50": p50, "p99": p99, "max": step_sorted[-1],
                       "buffer_ms": 2048 * frames / SR * 1000.0,
                       "meets_deadline": p99 < 2048 * frames / SR * 1000.0},
        # real-time factor (section 4.1): processing time / audio duration, of
        # one step of the whole batch and per stream
        "rtf": {"step": (total_ms / args.steps) / (2048 * frames / SR * 1000.0),
                "per_stream": (total_ms / args.steps) / (2048 * frames / SR * 1000.0) / streams},
        "e2e": {"value": e2e_value, "unit": "streams",
                "h2d_bytes_per_step": int(zh.numel() * 4), "d2h_bytes_per_step": int(yh.numel() * 4)},
        "roofline": roof,
        "roofline_other_kernels": roof_others,
        "fp32_same_batch": fp32_cmp,
        "memory": memory,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, d = oracle_sample(64, kind=kind)
        line["cpu_baseline"] = {"value": v, "unit": "streams", "cores": 1, "kind": "oracle",
                                "sample": f"1 stream x 64 buffers of 2048 samples, FP64 NumPy, "
                                          f"1 BLAS thread ({d['wall']:.1f} s)"}
        # the same sample with one BLAS thread per host core
        ncores = os.cpu_count() or 1
        v_all, d_all = oracle_sample(64, kind=kind, threads=ncores)
        line["cpu_baseline_all_cores"] = {"value": v_all, "unit": "streams", "cores": ncores, "kind": "oracle",
                                          "sample": f"as cpu_baseline with {ncores} BLAS threads "
                                                    f"({d_all['wall']:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
