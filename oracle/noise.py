"""SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator.

SplitMix64 keeps a 64-bit state that advances by the odd constant
GAMMA = 0x9E3779B97F4A7C15 and outputs a bijective mix of the new state.  Its
n-th output (n = 1, 2, ...) from initial state ``seed`` is therefore
``mix(seed + n * GAMMA)``, which lets any (stream, band, frame) draw its value
directly, independently of buffer boundaries.

Noise branch (RAVE's noise synthesiser, section 2.3, in the reduced
deterministic form used by this project): for band b of B bands and aligned
frame index t (the frame index of the *offline* model, so that the streamed and
offline outputs see the same noise),

    counter = t * B + b           (as an unsigned 64-bit integer)
    z       = mix(seed + (counter + 1) * GAMMA)
    u       = (z >> 40) * 2**-23 - 1        in [-1, 1), exact in float32.
"""
from __future__ import annotations

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB


def mix(z):
    """SplitMix64 output function (Steele, Lea & Flood 2014): the bijective mix of one state."""
    z &= MASK
    z = ((z ^ (z >> 30)) * MUL1) & MASK
    z = ((z ^ (z >> 27)) * MUL2) & MASK
    return z ^ (z >> 31)


def splitmix64_sequence(seed, count):
    """The first ``count`` outputs of a SplitMix64 generator seeded with
    ``seed`` (Steele, Lea & Flood 2014)."""
    state = seed & MASK
    out = []
    for _ in range(count):
        state = (state + GAMMA) & MASK
        out.append(mix(state))
    return out


def draw(seed, counter):
    """The (counter+1)-th SplitMix64 output from ``seed`` (the counter form of
    Steele, Lea & Flood 2014); counter may be negative."""
    return mix((seed + ((counter + 1) & MASK) * GAMMA) & MASK)


def uniform(seed, band, frame, bands):
    """u in [-1, 1) for one band and aligned frame: the heads' noise of section
    2.3, in this project's deterministic reading."""
    z = draw(seed, frame * bands + band)
    return (z >> 40) * 2.0 ** -23 - 1.0


def uniform_block(seed, t0, count, bands):
    """u[t, b] for frames t0 .. t0+count-1 (frames may be negative), float64:
    the heads' noise of section 2.3."""
    import numpy as np

    out = np.empty((count, bands))
    for i in range(count):
        for b in range(bands):
            out[i, b] = uniform(seed, b, t0 + i, bands)
    return out
