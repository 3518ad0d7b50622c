"""Latent manipulation of a streamed model's input (section 5.1, Fig. 7; section 5.2).

TEST INFRASTRUCTURE ONLY (see the package header).

Section 5.1 shows the first dimension of a decoder's latent biased and the last
one replaced by a user value while the model streams; section 5.2 offers a
scale, a bias and a random noise for each latent dimension.  The oracle writes
that per-frame, per-channel map out directly:

    x'[t, c] = scale[t, c] * x[t, c] + bias[t, c] + amp[t, c] * u(t, c)

Replacing dimension c by v is scale = 0, bias = v.  The paper leaves the
noise's law open; this project reads it as uniform in [-amp, amp), drawn by the
counter-based SplitMix64 generator of ``noise`` (the heads' generator) from the
seed ``stream_seed XOR TAG`` with counter t * channels + c.  Keying by the input
frame index t makes the streamed and the offline runs see the same values.
Parameters may change between buffers: they are given per frame.
"""
from __future__ import annotations

import numpy as np

from . import noise as N

# separates the input noise from the heads' noise of the same stream seed
TAG = 0x6C6174656E742D6E


def input_noise(seed, t0, count, channels):
    """u(t, c) for input frames t0 .. t0+count-1, float64 [count][channels]:
    section 5.2's per-dimension random noise, in this project's reading
    (uniform, SplitMix64 counter t * channels + c, tagged seed)."""
    s = (seed ^ TAG) & N.MASK
    out = np.empty((count, channels))
    for i in range(count):
        for c in range(channels):
            out[i, c] = N.uniform(s, c, t0 + i, channels)
    return out


def manipulate(x, scale=1.0, bias=0.0, amp=0.0, seed=0, t0=0):
    """The manipulated input frames (Fig. 7's bias and replacement, section
    5.1; section 5.2's scale, bias and noise).  x: [T][C]; scale, bias, amp
    broadcast to [T][C] (per frame and channel); t0 = index of x's first frame
    in the stream."""
    x = np.asarray(x, dtype=np.float64)
    T, C = x.shape
    scale = np.broadcast_to(np.asarray(scale, dtype=np.float64), (T, C))
    bias = np.broadcast_to(np.asarray(bias, dtype=np.float64), (T, C))
    amp = np.broadcast_to(np.asarray(amp, dtype=np.float64), (T, C))
    out = scale * x + bias
    if np.any(amp != 0):
        out = out + amp * input_noise(seed, t0, T, C)
    return out


def piecewise(T, C, changes, default):
    """A [T][C] parameter array that holds ``default`` until the first change;
    ``changes`` = [(frame, value [C] or scalar), ...] in frame order, each value
    held from its frame on: the real-time interaction of section 5.1, a user's
    control reaching the stream between buffers."""
    out = np.empty((T, C))
    out[:] = default
    for f, v in changes:
        out[f:] = v
    return out
