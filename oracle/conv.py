"""Eq. 1 convolution, padding, stride, dilation and transposed convolution (section 2.1).

Arrays follow the paper's notation: a signal is x in R^{M x T} (channels first),
a kernel is omega in R^{N x M x K}.  Transposed-convolution kernels use the
trained layout [C_in][C_out][K].
"""
from __future__ import annotations

import numpy as np

LEAKY_SLOPE = 0.2


def leaky_relu(x):
    """LeakyReLU with slope 0.2 (the activation of the RAVE-like workloads, section 2.3)."""
    return np.where(x >= 0, x, LEAKY_SLOPE * x)


def activate(x, act):
    """The layer input's activation, none or LeakyReLU (section 2.3's RAVE-like layers)."""
    if act is None:
        return x
    if act == "leaky":
        return leaky_relu(x)
    raise ValueError(f"unknown activation {act!r}")


def zero_pad(x, left, right):
    """Left / right zero padding along time (section 2.1)."""
    m, t = x.shape
    out = np.zeros((m, left + t + right), dtype=np.float64)
    out[:, left:left + t] = x
    return out


def correlate(x, w, stride=1, dilation=1):
    """Eq. 1 on an already padded input, generalised to stride S and dilation d:

        y^n[i] = sum_m sum_k w^{n,m}[k] x^m[i*S + k*d]

    for every i with i*S + (K-1)*d < T ("valid" outputs).  One tensordot per tap.
    """
    n_out, m_in, k = w.shape
    m, t = x.shape
    assert m == m_in, (m, m_in)
    span = (k - 1) * dilation
    if t <= span:
        return np.zeros((n_out, 0))
    count = (t - span - 1) // stride + 1
    y = np.zeros((n_out, count))
    for kk in range(k):
        start = kk * dilation
        cols = x[:, start:start + (count - 1) * stride + 1:stride]
        y += np.tensordot(w[:, :, kk], cols, axes=([1], [0]))
    return y


def correlate_loops(x, w, stride=1, dilation=1):
    """Eq. 1 written as the literal quadruple sum (tiny inputs only)."""
    n_out, m_in, k = w.shape
    t = x.shape[1]
    span = (k - 1) * dilation
    count = 0 if t <= span else (t - span - 1) // stride + 1
    y = np.zeros((n_out, count))
    for n in range(n_out):
        for i in range(count):
            acc = 0.0
            for m in range(m_in):
                for kk in range(k):
                    acc += w[n, m, kk] * x[m, i * stride + kk * dilation]
            y[n, i] = acc
    return y


def conv1d(x, w, b=None, stride=1, dilation=1, pad_left=0, pad_right=0):
    """Zero-padded convolution layer: pad, then Eq. 1, then add the bias."""
    y = correlate(zero_pad(x, pad_left, pad_right), w, stride, dilation)
    if b is not None:
        y = y + b[:, None]
    return y


def conv_transpose_full(x, w, stride):
    """Transposed convolution of section 2.1, full output (no crop):

        y^n[q*S + k] += sum_m w^{m,n}[k] x^m[q],   length (T-1)*S + K.

    Written as its scatter definition, one tensordot per tap.
    """
    m_in, n_out, k = w.shape
    m, t = x.shape
    assert m == m_in
    y = np.zeros((n_out, (t - 1) * stride + k if t > 0 else 0))
    if t == 0:
        return y
    for kk in range(k):
        contrib = np.tensordot(w[:, :, kk], x, axes=([0], [0]))  # [n_out][T]
        y[:, kk:kk + (t - 1) * stride + 1:stride] += contrib
    return y


def conv_transpose_full_loops(x, w, stride):
    """Section 2.1's transposed convolution by its scatter definition, as explicit
    loops (tiny inputs only)."""
    m_in, n_out, k = w.shape
    t = x.shape[1]
    y = np.zeros((n_out, (t - 1) * stride + k))
    for q in range(t):
        for m in range(m_in):
            for n in range(n_out):
                for kk in range(k):
                    y[n, q * stride + kk] += w[m, n, kk] * x[m, q]
    return y
