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


def causal_forward(nodes, params_t, x, seed=0, noise_on=True):
    """The causal model of section 3 in torch float64, for autograd.

    x: torch float64 [C][T]; params_t: {node: (w, b)} torch float64 tensors.
    Returns the last node's output [C_out][T_out]."""
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


def gradients(nodes, params, x, weight_out, seed=0, noise_on=True):
    """Offline gradients of the causal model (section 3), the reference for
    the chunked backward.  Loss L = sum(weight_out * y) over the causal model's output y
    ([T_out][C_out], channels-last like the library).  Returns (L, dL/dx as
    [T][C], {node: (dL/dw, dL/db)}) in float64 numpy."""
    xt = torch.tensor(np.asarray(x, np.float64).T.copy(), requires_grad=True)
    pt = {}
    for i, (w, b) in params.items():
        pt[i] = (torch.tensor(np.asarray(w, np.float64), requires_grad=True),
                 None if b is None else torch.tensor(np.asarray(b, np.float64), requires_grad=True))
    y = causal_forward(nodes, pt, xt, seed, noise_on)
    loss = (y * torch.tensor(np.asarray(weight_out, np.float64).T.copy())).sum()
    loss.backward()
    grads = {i: (w.grad.numpy().copy(), None if b is None else b.grad.numpy().copy()) for i, (w, b) in pt.items()}
    return float(loss.detach()), xt.grad.numpy().T.copy(), grads
