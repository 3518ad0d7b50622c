"""Seeded synthetic workloads: layer lists, random weights and input signals.

This module is the one piece shared by the CUDA path and the FP64 oracle.  It
holds no arithmetic of the streaming method: it only *describes* models (plain
lists of node dictionaries, exactly what a caller hands to ``cc_model_create``)
and draws seeded random numbers.  Delays, caches, convolutions and filter-bank
designs live on each side separately.

Node dictionary fields (all integers unless noted):

``op``        ``"input" | "conv" | "convt" | "add" | "heads"``
``inputs``    list of producer node indices (topological order: all < own index)
``c_in``      input channels (``input``: the model's input channels)
``c_out``     output channels
``k``         kernel size K (conv / convt)
``stride``    stride S (conv: downsampling; convt: upsampling)
``dilation``  dilation d (conv only)
``pad_left``  left zero padding of the *trained* (offline) layer, in input frames
``pad_right`` right zero padding of the trained layer, in input frames
``crop``      left crop p of a transposed convolution's full output (the trained
              layer crops ``p`` on the left and ``K - S - p`` on the right)
``act_in``    ``"leaky"`` (LeakyReLU, slope 0.2, applied to the node's input) or None
``bias``      bool

The ``heads`` node combines three equally sized branches (waveform, amplitude,
noise) as ``tanh(w) * sigmoid(a) + sigmoid(n) * u`` where ``u`` is a seeded
counter-based noise in [-1, 1) (RAVE's noise synthesiser, section 2.3, reduced to
a deterministic form so that streamed and offline outputs can be compared).

Paper: Caillon & Esling, "Streamable neural audio synthesis with non-causal
convolutions" (DAFx-22).  The RAVE-like layouts follow section 2.3 (strided
convolutional encoder, residual transposed-convolutional decoder, noise
synthesiser); the widths, ratios, kernel sizes and PQMF sizes are the workload
definitions of this project (48 kHz, 16-band PQMF with 64 taps).
"""
from __future__ import annotations

import numpy as np

LEAKY = "leaky"


def _node(op, inputs, c_in, c_out, k=1, stride=1, dilation=1, pad_left=0,
          pad_right=0, crop=0, act_in=None, bias=True, name=""):
    return dict(op=op, inputs=list(inputs), c_in=int(c_in), c_out=int(c_out),
                k=int(k), stride=int(stride), dilation=int(dilation),
                pad_left=int(pad_left), pad_right=int(pad_right), crop=int(crop),
                act_in=act_in, bias=bool(bias), name=name)


def input_node(channels, name="input"):
    return _node("input", [], channels, channels, bias=False, name=name)


def tiny_stack(channels=16, kernel=3, dilations=(1, 2, 4)):
    """Three non-causal dilated Conv1d layers, LeakyReLU(0.2) between layers.

    Each layer is "same"-padded symmetrically: pad (K-1)*d/2 frames on each side
    (section 2.1: padding K-1 zeros keeps the temporal length).
    """
    nodes = [input_node(channels)]
    for i, d in enumerate(dilations):
        half = (kernel - 1) * d // 2
        nodes.append(_node("conv", [len(nodes) - 1], channels, channels, k=kernel,
                           dilation=d, pad_left=half, pad_right=(kernel - 1) * d - half,
                           act_in=LEAKY if i > 0 else None, name=f"conv{i}"))
    return nodes


def rave_decoder(latent=128, capacity=64, ratios=(4, 4, 4, 2), dilations=(1, 3, 9),
                 bands=16, pqmf_taps=64, head_kernels=(7, 3, 3)):
    """RAVE-like residual transposed-convolutional decoder + 16-band inverse PQMF.

    pre:   Conv(latent -> C0, k=3, pad 1/1), C0 = capacity * 2**len(ratios)
    stage: LeakyReLU -> ConvT(C -> C/2, K=2r, S=r, crop r/2), then residual
           units with dilations d: LeakyReLU -> Conv(k=3, dil d, pad d/d)
           -> LeakyReLU -> Conv(k=1) -> + skip
    heads: waveform Conv(k=7, pad 3/3), amplitude Conv(k=3, pad 1/1), noise
           Conv(k=3) -> LeakyReLU -> Conv(k=3), all on LeakyReLU(h), each to
           ``bands`` channels; combined by the ``heads`` node
    PQMF:  inverse PQMF as ConvT(bands -> 1, K=pqmf_taps, S=bands,
           crop (K - S)/2), no bias; its weights are the synthesis filters
           (filled in by the caller, see ``pqmf_node_index``).
    """
    nodes = [input_node(latent)]
    c = capacity * 2 ** len(ratios)
    nodes.append(_node("conv", [0], latent, c, k=3, pad_left=1, pad_right=1, name="pre"))
    for si, r in enumerate(ratios):
        nodes.append(_node("convt", [len(nodes) - 1], c, c // 2, k=2 * r, stride=r,
                           crop=r // 2, act_in=LEAKY, name=f"up{si}"))
        c //= 2
        for d in dilations:
            skip = len(nodes) - 1
            nodes.append(_node("conv", [skip], c, c, k=3, dilation=d, pad_left=d,
                               pad_right=d, act_in=LEAKY, name=f"s{si}d{d}a"))
            nodes.append(_node("conv", [len(nodes) - 1], c, c, k=1, act_in=LEAKY,
                               name=f"s{si}d{d}b"))
            nodes.append(_node("add", [skip, len(nodes) - 1], c, c, bias=False,
                               name=f"s{si}d{d}add"))
    h = len(nodes) - 1
    kw, ka, kn = head_kernels
    nodes.append(_node("conv", [h], c, bands, k=kw, pad_left=kw // 2, pad_right=kw // 2,
                       act_in=LEAKY, name="wave"))
    wave = len(nodes) - 1
    nodes.append(_node("conv", [h], c, bands, k=ka, pad_left=ka // 2, pad_right=ka // 2,
                       act_in=LEAKY, name="amp"))
    amp = len(nodes) - 1
    nodes.append(_node("conv", [h], c, bands, k=kn, pad_left=kn // 2, pad_right=kn // 2,
                       act_in=LEAKY, name="noise1"))
    nodes.append(_node("conv", [len(nodes) - 1], bands, bands, k=kn, pad_left=kn // 2,
                       pad_right=kn // 2, act_in=LEAKY, name="noise2"))
    noise = len(nodes) - 1
    nodes.append(_node("heads", [wave, amp, noise], bands, bands, bias=False, name="heads"))
    nodes.append(_node("convt", [len(nodes) - 1], bands, 1, k=pqmf_taps, stride=bands,
                       crop=(pqmf_taps - bands) // 2, bias=False, name="ipqmf"))
    return nodes


def rave_encoder(latent=128, capacity=64, ratios=(4, 4, 4, 2), bands=16, pqmf_taps=64):
    """RAVE-like strided convolutional encoder with a 16-band PQMF analysis front end.

    PQMF:  Conv(1 -> bands, K=pqmf_taps, S=bands, pad (K-S)/2 both sides), no bias;
           its weights are the analysis filters (filled in by the caller)
    conv:  Conv(bands -> capacity, k=7, pad 3/3)
    stage: LeakyReLU -> Conv(C -> 2C, K=2r+1, S=r, pad r/r)
    out:   LeakyReLU -> Conv(C -> latent, k=3, pad 1/1) (the latent mean; the
           encoder variance is set to 0 as in section 4.2)
    """
    nodes = [input_node(1)]
    half = (pqmf_taps - bands) // 2
    nodes.append(_node("conv", [0], 1, bands, k=pqmf_taps, stride=bands, pad_left=half,
                       pad_right=half, bias=False, name="pqmf"))
    nodes.append(_node("conv", [1], bands, capacity, k=7, pad_left=3, pad_right=3, name="in"))
    c = capacity
    for si, r in enumerate(ratios):
        nodes.append(_node("conv", [len(nodes) - 1], c, 2 * c, k=2 * r + 1, stride=r,
                           pad_left=r, pad_right=r, act_in=LEAKY, name=f"down{si}"))
        c *= 2
    nodes.append(_node("conv", [len(nodes) - 1], c, latent, k=3, pad_left=1, pad_right=1,
                       act_in=LEAKY, name="mean"))
    return nodes


def pqmf_node_index(nodes):
    """Index of the PQMF layer (named ``ipqmf`` or ``pqmf``), or None."""
    for i, n in enumerate(nodes):
        if n["name"] in ("ipqmf", "pqmf"):
            return i
    return None


def weight_shape(node):
    """Trained-layer weight layout: conv [C_out][C_in][K]; convt [C_in][C_out][K]."""
    if node["op"] == "conv":
        return (node["c_out"], node["c_in"], node["k"])
    if node["op"] == "convt":
        return (node["c_in"], node["c_out"], node["k"])
    return None


def fan_in(node):
    if node["op"] == "conv":
        return node["c_in"] * node["k"]
    if node["op"] == "convt":
        return node["c_in"] * node["k"] // node["stride"]
    return 1


def init_params(nodes, seed, dtype=np.float64):
    """Weights and biases ~ N(0, 1/fan_in) from ``seed`` (fan_in = C_in*K, or
    C_in*K/S for a transposed convolution).  Returns {node index: (w, b)}."""
    rng = np.random.default_rng(seed)
    params = {}
    for i, n in enumerate(nodes):
        shp = weight_shape(n)
        if shp is None:
            continue
        std = 1.0 / np.sqrt(fan_in(n))
        w = rng.standard_normal(shp) * std
        b = rng.standard_normal(n["c_out"]) * std if n["bias"] else None
        params[i] = (w.astype(dtype), None if b is None else b.astype(dtype))
    return params


def identity_params(nodes):
    """Weights that make every layer an identity (or nearest-neighbour upsampler)
    in the *trained* (non-causal) model: a conv's one-hot tap sits where the
    trained padding centres the kernel (tap k with k*d == pad_left), a transposed
    convolution repeats each input frame S times after its crop, biases are zero.
    Used with ``act_in`` removed, such a model is the identity, so its causal
    reconfiguration must be a pure delay."""
    params = {}
    for i, n in enumerate(nodes):
        shp = weight_shape(n)
        if shp is None:
            continue
        w = np.zeros(shp)
        if n["op"] == "conv":
            tap = n["pad_left"] // n["dilation"]
            for c in range(min(n["c_in"], n["c_out"])):
                w[c, c, tap] = 1.0
        else:
            p, s = n["crop"], n["stride"]
            for c in range(min(n["c_in"], n["c_out"])):
                w[c, c, p:p + s] = 1.0
        params[i] = (w, np.zeros(n["c_out"]) if n["bias"] else None)
    return params


def strip_activations(nodes):
    return [dict(n, act_in=None) for n in nodes]


def signal(seed, frames, channels, std=1.0):
    """Channels-last white noise [frames][channels] ~ N(0, std^2)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((frames, channels)) * std


def stream_seeds(seed, count):
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.integers(0, 2 ** 63 - 1, size=count, dtype=np.int64)]


def buffer_partition(total, seed, choices):
    """A random partition of ``total`` frames into buffers drawn from ``choices``
    (the last buffer takes the remainder)."""
    rng = np.random.default_rng(seed)
    parts, left = [], total
    while left > 0:
        b = int(rng.choice(choices))
        b = min(b, left)
        parts.append(b)
        left -= b
    return parts


def chain(first, second):
    """One layer list feeding ``first``'s last node into ``second`` (whose input
    node is dropped): e.g. encoder then decoder, an audio -> audio model."""
    off = len(first) - 1  # second's node k (k >= 1) becomes node off + k
    out = [dict(n) for n in first]
    for n in second[1:]:
        m = dict(n)
        m["inputs"] = [off if u == 0 else off + u for u in n["inputs"]]
        out.append(m)
    return out
