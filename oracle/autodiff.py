"""Gradients of the causally reconfigured model (reference for the backward pass).

TEST INFRASTRUCTURE ONLY (see the package header).  The causal offline model
of section 3 (all trained padding moved to the left, Eq. 2 extra delays before
strided layers, Eq. 3 delays on merged branches, no left crop on transposed
convolutions) written with torch float64 CPU operators, so that the library
routine torch.autograd provides its gradients with respect to the input, the
weights and the biases.  It shares no code with the numpy forms in
``model.py``; the two are checked against each other and against finite
differences in the test suite.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

from . import model as M
from . import noise as N


def _act(x, act):
    return F.leaky_relu(x, 0.2) if act == "leaky" else x


_LP = {"bf16": torch.bfloat16, "f16": torch.float16}


def round_to(v, fmt):
    """v (float64) rounded to the nearest `fmt` number, ties to even, through
    float32 (the accumulator type whose values a low-precision layer stores):
    "bf16" keeps 8 significant bits, "f16" 11.  torch's casts do the rounding."""
    return v.to(torch.float32).to(_LP[fmt]).to(torch.float64)


def round_weights(w, fmt, op, stride=1):
    """The weights a rounded layer multiplies (float64 in, float64 out): each
    GEMM row is scaled to max |w| = 1 in float32, rounded with round_to, and
    multiplied back by its float32 scale.  A convolution's row is one output
    channel over (input channel, tap); a transposed convolution's row is one
    output channel and one output phase ph over the input channels and the
    taps k = ph + j*stride that write that phase (a row of zeros keeps scale 1)."""
    w32 = w.to(torch.float32)
    mag = w32.abs()
    if op == "conv":
        sc = mag.amax(dim=(1, 2), keepdim=True).expand_as(w32).clone()
    else:
        sc = torch.empty_like(w32)
        for ph in range(stride):
            sc[:, :, ph::stride] = mag[:, :, ph::stride].amax(dim=(0, 2), keepdim=True)
    sc = torch.where(sc > 0, sc, torch.ones_like(sc))
    q = round_to((w32 / sc).to(torch.float64), fmt)
    return q * sc.to(torch.float64)


def _rounded_w(w, fmt, op, stride):
    """round_weights in the forward, the identity in the backward."""
    return w + (round_weights(w.detach(), fmt, op, stride) - w.detach())


def _rounded(v, fmt):
    """round_to(v) in the forward, the identity in the backward: the gradient
    of a layer that multiplies rounded operands, taken with respect to the
    values before rounding (the rounding's derivative is taken as 1)."""
    return v + (round_to(v.detach(), fmt) - v.detach())


def causal_forward(nodes, params_t, x, seed=0, noise_on=True, rounded=None):
    """The causal model of section 3 in torch float64, for autograd.

    x: torch float64 [C][T]; params_t: {node: (w, b)} torch float64 tensors.
    rounded: {node: "bf16" | "f16"} for convolutions that multiply their
    activated input rounded to that type (round_to) and their weights rounded
    row by row (round_weights); bias, accumulation and every other value stay
    exact.  Returns the last node's output
    [C_out][T_out]."""
    rounded = rounded or {}
    info = M.analyze(nodes)
    vals = []
    for i, nd in enumerate(nodes):
        op = nd["op"]
        if op == "input":
            vals.append(x)
            continue
        if op in ("conv", "convt"):
            w, b = params_t[i]
            a = _act(vals[nd["inputs"][0]], nd["act_in"])[None]
            if i in rounded:
                a = _rounded(a, rounded[i])
                w = _rounded_w(w, rounded[i], op, nd["stride"])
            t_in = a.shape[-1]
            s = nd["stride"]
            if op == "conv":
                left = nd["pad_left"] + nd["pad_right"] + info["Da"][i]
                y = F.conv1d(F.pad(a, (left, 0)), w, b, stride=s, dilation=nd["dilation"])[0]
                y = y[:, :t_in // s]
            else:
                y = F.conv_transpose1d(a, w, None, stride=s)[0][:, :t_in * s]
                if b is not None:
                    y = y + b[:, None]
            vals.append(y)
            continue
        ins = []
        for u, a in zip(nd["inputs"], info["A"][i]):
            v = vals[u]
            ins.append(F.pad(v, (a, 0))[:, :v.shape[1]] if a else v)
        if op == "add":
            vals.append(ins[0] + ins[1])
        else:
            y = torch.tanh(ins[0]) * torch.sigmoid(ins[1])
            if noise_on:
                bands, t = ins[0].shape
                u = torch.from_numpy(N.uniform_block(seed, -info["D"][i], t, bands).T.copy())
                y = y + torch.sigmoid(ins[2]) * u
            vals.append(y)
    return vals[-1]


def gradients(nodes, params, x, weight_out, seed=0, noise_on=True, rounded=None):
    """Offline gradients of the causal model (section 3), the reference for
    the chunked backward.  Loss L = sum(weight_out * y) over the causal model's output y
    ([T_out][C_out], channels-last like the library).  `rounded` as in
    causal_forward: the gradients are then those of the model with rounded
    operands (the weight gradient of a rounded layer is with respect to its
    weights before rounding).  Returns (L, dL/dx as [T][C], {node: (dL/dw,
    dL/db)}) in float64 numpy."""
    xt = torch.tensor(np.asarray(x, np.float64).T.copy(), requires_grad=True)
    pt = {}
    for i, (w, b) in params.items():
        pt[i] = (torch.tensor(np.asarray(w, np.float64), requires_grad=True),
                 None if b is None else torch.tensor(np.asarray(b, np.float64), requires_grad=True))
    y = causal_forward(nodes, pt, xt, seed, noise_on, rounded)
    loss = (y * torch.tensor(np.asarray(weight_out, np.float64).T.copy())).sum()
    loss.backward()
    grads = {i: (w.grad.numpy().copy(), None if b is None else b.grad.numpy().copy()) for i, (w, b) in pt.items()}
    return float(loss.detach()), xt.grad.numpy().T.copy(), grads
