"""Post-training causal reconfiguration, offline models and cached-padding streaming.

A model is a list of node dictionaries (see the field list in the package's
workload module: op, inputs, c_in, c_out, k, stride, dilation, pad_left,
pad_right, crop, act_in, bias) plus ``params = {node: (w, b)}``.  Signals at
this file's API are channels-last [T][C]; internally the paper's [C][T].

Paper passages restated here:

* section 3: the trained layer's right padding R becomes extra left padding,
  so every layer turns causal and its output is delayed by R.
* section 3.1: strided convolutions get an extra input delay D_a so that the
  cumulated lag D_c + R + D_a is a multiple of the stride S (Eq. 2); transposed
  and stride-1 convolutions only delay their output; the cumulated lag is
  carried layer by layer.
* section 3.2, Eq. 3: at a merge of parallel branches with cumulated delays
  D_i, branch i is delayed by A_i = max_j D_j - D_i.
* Fig. 1 / section 2.2: cached padding keeps the last N input frames of a
  buffer and prepends them to the next buffer, N being the layer's (now
  entirely left) padding.
* section 4.2: once latency is compensated the streamed output equals the
  offline one.
"""
from __future__ import annotations

from fractions import Fraction
from math import gcd

import numpy as np

from . import conv as C
from . import noise as N


# ----------------------------------------------------------------------------
# Eq. 2 / Eq. 3 delay analysis
# ----------------------------------------------------------------------------

def stride_alignment(stride, right_pad, cumulated):
    """Eq. 2: extra input delay D_a making D_c + R + D_a a multiple of S.

    The printed formula "S - (R + D_c mod S) mod S" is read with the minimal
    result: D_a = (S - ((R + D_c) mod S)) mod S, in [0, S).
    """
    return (stride - ((right_pad + cumulated) % stride)) % stride


def analyze(nodes):
    """Per-node causal-reconfiguration numbers.

    Returns a dict of lists indexed by node:
      rate  Fraction, frames of this node per input frame
      D     cumulated delay at the node's output, in the node's own frames
      Da    Eq. 2 extra delay (conv nodes), else 0
      A     Eq. 3 per-input alignment delays (merge nodes), else []
      H     frames of input history a node needs from each producer (the
            cached padding length): conv pL + pR + Da; convt ceil(K/S) - 1;
            merges A_i
    and the scalars ``delay`` (output node, output frames) and
    ``in_per_step`` (smallest input length giving whole frames everywhere).
    """
    n = len(nodes)
    rate = [Fraction(0)] * n
    D = [0] * n
    Da = [0] * n
    A = [[] for _ in range(n)]
    for i, nd in enumerate(nodes):
        op = nd["op"]
        if op == "input":
            rate[i] = Fraction(1)
            D[i] = 0
        elif op == "conv":
            u = nd["inputs"][0]
            s = nd["stride"]
            rate[i] = rate[u] / s
            Da[i] = stride_alignment(s, nd["pad_right"], D[u])
            total = D[u] + nd["pad_right"] + Da[i]
            assert total % s == 0
            D[i] = total // s
        elif op == "convt":
            u = nd["inputs"][0]
            rate[i] = rate[u] * nd["stride"]
            D[i] = D[u] * nd["stride"] + nd["crop"]
        elif op in ("add", "heads"):
            ds = [D[u] for u in nd["inputs"]]
            rs = {rate[u] for u in nd["inputs"]}
            assert len(rs) == 1, "merged branches must run at one rate"
            rate[i] = rs.pop()
            D[i] = max(ds)
            A[i] = [D[i] - d for d in ds]
        else:
            raise ValueError(op)
    in_per_step = 1
    for r in rate:
        den = r.denominator
        in_per_step = in_per_step * den // gcd(in_per_step, den)
    return dict(rate=rate, D=D, Da=Da, A=A, delay=D[-1], in_per_step=in_per_step)


def history(nodes, info):
    """Cached-padding length each consumer needs from each of its inputs (the
    cached padding of section 2.2 with Eq. 2's extra delay)."""
    hist = []
    for i, nd in enumerate(nodes):
        op = nd["op"]
        if op == "conv":
            hist.append([nd["pad_left"] + nd["pad_right"] + info["Da"][i]])
        elif op == "convt":
            hist.append([-(-nd["k"] // nd["stride"]) - 1])
        elif op in ("add", "heads"):
            hist.append(list(info["A"][i]))
        else:
            hist.append([])
    return hist


def cache_frames(nodes, info):
    """Per node (section 2.2's cache): frames of its output kept between buffers (max over consumers)."""
    keep = [0] * len(nodes)
    for i, (nd, hs) in enumerate(zip(nodes, history(nodes, info))):
        for u, h in zip(nd["inputs"], hs):
            keep[u] = max(keep[u], h)
    return keep


def cache_elements(nodes, info):
    """Closed-form streaming state size: sum over nodes of kept frames x
    channels (section 4.1 reports this memory as the method's only overhead)."""
    keep = cache_frames(nodes, info)
    return sum(k * nd["c_out"] for k, nd in zip(keep, nodes))


def warmup_frames(nodes):
    """The start-up boundary effect of section 4.2's comparison.  Leading output
    frames of the offline original that the causal model may
    not reproduce (the paper compensates latency but does not discuss this
    start-up effect).  An inner layer's left zero padding at negative times is
    replaced, in the causal model, by that layer's pre-roll output; a frame is
    exact once none of its inputs reaches into such a region.  For weights with
    no zero tap (random weights) the count is tight: the frame just before it
    differs."""
    n = len(nodes)
    bad = [0] * n
    zneg = [False] * n  # causal values at negative (original) times are zero
    for i, nd in enumerate(nodes):
        op = nd["op"]
        if op == "input":
            bad[i], zneg[i] = 0, True
        elif op == "conv":
            u = nd["inputs"][0]
            s = nd["stride"]
            if zneg[u] and bad[u] == 0:
                bad[i] = 0
            else:
                bad[i] = -(-(bad[u] + nd["pad_left"]) // s)
            zneg[i] = zneg[u] and not nd["bias"]
        elif op == "convt":
            u = nd["inputs"][0]
            s, k, p = nd["stride"], nd["k"], nd["crop"]
            if zneg[u] and bad[u] == 0:
                bad[i] = 0
            else:
                # full-output index f sums inputs q with 0 <= f - q*s < k; it is
                # exact once its first input, ceil((f - k + 1) / s), is past the
                # bad region: f >= s*bad[u] - s + k, i.e. cropped t >= that - p
                bad[i] = max(0, bad[u] * s - s + k - p)
            zneg[i] = zneg[u] and not nd["bias"]
        elif op == "add":
            bad[i] = max(bad[u] for u in nd["inputs"])
            zneg[i] = all(zneg[u] for u in nd["inputs"])
        elif op == "heads":
            bad[i] = max(bad[u] for u in nd["inputs"])
            zneg[i] = False
    return bad[-1]


# ----------------------------------------------------------------------------
# Node arithmetic shared by the two offline forms
# ----------------------------------------------------------------------------

def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def heads_combine(wave, amp, noise_logit, seed, t0, noise_on=True):
    """RAVE-like output combination (section 2.3's heads with the noise
    synthesiser): tanh(wave) * sigmoid(amp) + sigmoid(noise) * u,
    u drawn for aligned frames t0, t0+1, ... ([C][T] arrays)."""
    y = np.tanh(wave) * _sigmoid(amp)
    if noise_on:
        bands, t = wave.shape
        u = N.uniform_block(seed, t0, t, bands).T
        y = y + _sigmoid(noise_logit) * u
    return y


def _delay(x, a):
    """Delay by a frames with zero fill, keeping the length."""
    if a == 0:
        return x
    out = np.zeros_like(x)
    out[:, a:] = x[:, :x.shape[1] - a] if x.shape[1] > a else 0.0
    return out


# ----------------------------------------------------------------------------
# Offline forms
# ----------------------------------------------------------------------------

def run_offline(nodes, params, x, causal, seed=0, noise_on=True):
    """Whole-signal evaluation.  ``causal=False``: the trained non-causal model
    (every layer padded pL left / pR right, transposed convolutions cropped p
    left and K-S-p right).  ``causal=True``: the post-training reconfiguration
    (section 3): all padding on the left, plus Eq. 2's D_a on strided layers,
    no crop on the left of transposed convolutions (output truncated to T*S),
    and Eq. 3 delays on merged branches.  x: [T][C_in]; returns [T_out][C_out]."""
    info = analyze(nodes)
    vals = []
    for i, nd in enumerate(nodes):
        op = nd["op"]
        if op == "input":
            vals.append(np.asarray(x, dtype=np.float64).T.copy())
            continue
        if op in ("conv", "convt"):
            w, b = params[i]
            a = C.activate(vals[nd["inputs"][0]], nd["act_in"])
            t_in = a.shape[1]
            s = nd["stride"]
            if op == "conv":
                if causal:
                    y = C.conv1d(a, w, b, s, nd["dilation"],
                                 nd["pad_left"] + nd["pad_right"] + info["Da"][i], 0)
                    y = y[:, :t_in // s]
                else:
                    y = C.conv1d(a, w, b, s, nd["dilation"], nd["pad_left"], nd["pad_right"])
            else:
                full = C.conv_transpose_full(a, w, s)
                start = 0 if causal else nd["crop"]
                y = full[:, start:start + t_in * s]
                if b is not None:
                    y = y + b[:, None]
            vals.append(y)
            continue
        ins = [vals[u] for u in nd["inputs"]]
        if causal:
            ins = [_delay(v, a) for v, a in zip(ins, info["A"][i])]
        if op == "add":
            vals.append(sum(ins))
        elif op == "heads":
            t0 = -info["D"][i] if causal else 0
            vals.append(heads_combine(ins[0], ins[1], ins[2], seed, t0, noise_on))
        else:
            raise ValueError(op)
    return vals[-1].T.copy()


def run_original(nodes, params, x, seed=0, noise_on=True):
    """The original non-causal model offline (pads L/R, crops; Eq. 1, section 2.1)."""
    return run_offline(nodes, params, x, causal=False, seed=seed, noise_on=noise_on)


def run_causal(nodes, params, x, seed=0, noise_on=True):
    """The causally reconfigured model offline (section 3: all padding left, Eq. 2, Eq. 3)."""
    return run_offline(nodes, params, x, causal=True, seed=seed, noise_on=noise_on)


# ----------------------------------------------------------------------------
# Cached-padding streaming (Fig. 1), written independently of the offline forms
# ----------------------------------------------------------------------------

class Stream:
    """Buffer-by-buffer evaluation of the reconfigured model.

    Each convolution keeps the last N frames of its (activated) input, N being
    its total left padding after reconfiguration, and prepends them to the next
    buffer (Fig. 1); each merged branch keeps A_i frames (Eq. 3).  Caches start
    at zero, which is the zero left padding of the offline causal model.
    """

    def __init__(self, nodes, params, seed=0, noise_on=True):
        self.nodes = nodes
        self.params = params
        self.seed = seed
        self.noise_on = noise_on
        self.info = analyze(nodes)
        self.hist = history(nodes, self.info)
        self.caches = []
        for nd, hs in zip(nodes, self.hist):
            chans = [nodes[u]["c_out"] for u in nd["inputs"]]
            self.caches.append([np.zeros((c, h)) for c, h in zip(chans, hs)])
        self.frames_out = [0] * len(nodes)  # frames emitted so far, per node

    @property
    def in_per_step(self):
        """Smallest input length giving every layer whole frames (section 3.1's alignment)."""
        return self.info["in_per_step"]

    def _window(self, i, j, new):
        cache = self.caches[i][j]
        win = np.concatenate([cache, new], axis=1)
        h = cache.shape[1]
        self.caches[i][j] = win[:, win.shape[1] - h:].copy() if h else cache
        return win

    def process(self, buf):
        """One DSP call (section 1, Fig. 1).  buf: [n][C_in], n a multiple of
        in_per_step.  Returns [n_out][C_out]."""
        buf = np.asarray(buf, dtype=np.float64)
        if buf.shape[0] % self.in_per_step:
            raise ValueError("buffer length must be a multiple of in_per_step")
        outs = []
        for i, nd in enumerate(self.nodes):
            op = nd["op"]
            if op == "input":
                outs.append(buf.T.copy())
            elif op == "conv":
                w, b = self.params[i]
                new = C.activate(outs[nd["inputs"][0]], nd["act_in"])
                s = nd["stride"]
                win = self._window(i, 0, new)
                y = C.correlate(win, w, s, nd["dilation"])[:, :new.shape[1] // s]
                outs.append(y if b is None else y + b[:, None])
            elif op == "convt":
                w, b = self.params[i]
                new = C.activate(outs[nd["inputs"][0]], nd["act_in"])
                s = nd["stride"]
                h = self.hist[i][0]
                win = self._window(i, 0, new)
                full = C.conv_transpose_full(win, w, s)
                y = full[:, h * s:(h + new.shape[1]) * s]
                outs.append(y if b is None else y + b[:, None])
            else:
                aligned = []
                for j, u in enumerate(nd["inputs"]):
                    new = outs[u]
                    win = self._window(i, j, new)
                    aligned.append(win[:, :new.shape[1]])
                if op == "add":
                    outs.append(sum(aligned))
                else:
                    t0 = self.frames_out[i] - self.info["D"][i]
                    outs.append(heads_combine(aligned[0], aligned[1], aligned[2],
                                              self.seed, t0, self.noise_on))
            self.frames_out[i] += outs[-1].shape[1]
        return outs[-1].T.copy()

    def run(self, x, partition):
        """Stream x [T][C] through buffers of the given lengths and concatenate
        (section 4.2's buffer-size experiment)."""
        pieces, pos = [], 0
        for n in partition:
            pieces.append(self.process(x[pos:pos + n]))
            pos += n
        return np.concatenate(pieces, axis=0)
