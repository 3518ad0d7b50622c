"""Random streamable layer lists (seeded), CPU only.

For each graph, a chain of dilated convs, strided convs, transposed convs and
residual units (a branch conv added back to its input, Eq. 3 alignment), and
in half of them a final heads merge of three branches of different reach:

* the library's planning pass (a plan-only model, no GPU) reproduces the
  oracle's section 3 analysis node by node: cumulated delay, Eq. 2 extra
  delay, Eq. 3 alignments, kept cache frames, frames per model step, total
  delay and state size;
* the oracle's cached-padding stream equals its causal offline model on a
  random buffer partition (E1), and the causal model equals the original
  non-causal model delayed by the total delay on the interior (E2).

Trained layers are taken with "same"-style padding, (K - 1) x dilation zeros
split between left and right, as in the RAVE-like workloads."""
import numpy as np
import pytest

from oracle import model as M
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

SEEDS = list(range(40))


def random_graph(seed, channels=None):
    """The seeded layer list; `channels` overrides the drawn width (2, 3 or 4)
    with the same topology and geometry (for the tensor-core path)."""
    rng = np.random.default_rng(seed)
    C = int(rng.choice([2, 3, 4]))
    if channels is not None:
        C = channels
    nodes = [W.input_node(C)]

    def conv(src, k, d, s, name, act):
        span = (k - 1) * d
        left = int(rng.integers(0, span + 1))
        nodes.append(W._node("conv", [src], C, C, k=k, stride=s, dilation=d, pad_left=left,
                             pad_right=span - left, act_in=act, name=name))
        return len(nodes) - 1

    cur = 0
    for i in range(int(rng.integers(2, 7))):
        kind = rng.choice(["conv", "strided", "convt", "res"], p=[0.3, 0.2, 0.2, 0.3])
        act = W.LEAKY if (i > 0 and rng.random() < 0.5) else None
        if kind == "conv":
            cur = conv(cur, int(rng.integers(1, 6)), int(rng.integers(1, 4)), 1, f"c{i}", act)
        elif kind == "strided":
            s = int(rng.integers(2, 4))
            cur = conv(cur, int(rng.choice([s, 2 * s, 2 * s + 1])), 1, s, f"s{i}", act)
        elif kind == "convt":
            s = int(rng.integers(2, 4))
            k = s * int(rng.integers(1, 4))
            nodes.append(W._node("convt", [cur], C, C, k=k, stride=s, crop=int(rng.integers(0, k - s + 1)),
                                 act_in=act, name=f"t{i}"))
            cur = len(nodes) - 1
        else:
            b = conv(cur, int(rng.choice([1, 3, 5])), int(rng.integers(1, 4)), 1, f"r{i}", act)
            if rng.random() < 0.5:  # a two-conv branch
                b = conv(b, int(rng.choice([1, 3])), 1, 1, f"r{i}b", W.LEAKY)
            nodes.append(W._node("add", [cur, b], C, C, bias=False, name=f"add{i}"))
            cur = len(nodes) - 1
    if rng.random() < 0.5:
        # the heads merge: three branches of different reach (Eq. 3 over three
        # inputs; the noise is keyed on the aligned frame index)
        br = [conv(cur, int(rng.choice([1, 3, 5, 7])), int(rng.integers(1, 3)), 1, f"h{q}", W.LEAKY)
              for q in range(3)]
        if rng.random() < 0.5:
            br[2] = conv(br[2], 3, 1, 1, "h2b", W.LEAKY)
        nodes.append(W._node("heads", br, C, C, bias=False, name="heads"))
    return nodes


@pytest.mark.parametrize("seed", SEEDS)
def test_plan_matches_oracle_on_random_graphs(cclib, seed):
    nodes = random_graph(seed)
    info = M.analyze(nodes)
    keep = M.cache_frames(nodes, info)
    m = api.Model(nodes, {}, max_streams=0)
    assert m.total_delay == info["delay"]
    assert m.io["in_per_step"] == info["in_per_step"]
    for i, nd in enumerate(nodes):
        ni = m.node_info(i)
        assert ni["delay"] == info["D"][i], (seed, i, nd["name"])
        assert ni["extra_delay"] == info["Da"][i], (seed, i, nd["name"])
        assert ni["align"][:len(info["A"][i])] == info["A"][i], (seed, i, nd["name"])
        assert ni["kept"] == keep[i], (seed, i, nd["name"])
        assert ni["frames_per_step"] == info["rate"][i] * info["in_per_step"], (seed, i, nd["name"])
    assert m.state_bytes[0] == 4 * M.cache_elements(nodes, info)
    m.close()


@pytest.mark.parametrize("seed", SEEDS)
def test_oracle_stream_and_delay_on_random_graphs(seed):
    nodes = random_graph(seed)
    p = W.init_params(nodes, 100 + seed)
    info = M.analyze(nodes)
    step = info["in_per_step"]
    rng = np.random.default_rng(1000 + seed)
    n_steps = 12
    x = rng.standard_normal((step * n_steps, nodes[0]["c_out"]))
    y_causal = M.run_causal(nodes, p, x)
    # E1: streaming == causal offline, for a random partition into whole steps
    cuts, left = [], n_steps
    while left:
        n = int(rng.integers(1, min(left, 4) + 1))
        cuts.append(n * step)
        left -= n
    s = M.Stream(nodes, p)
    y_stream = s.run(x, cuts)
    np.testing.assert_allclose(y_stream, y_causal, rtol=0, atol=1e-12 * max(1.0, np.abs(y_causal).max()))
    # E2: causal[t + D] == original[t] on the interior [W, T_out - D)
    y_orig = M.run_original(nodes, p, x)
    D = info["delay"]
    Wu = M.warmup_frames(nodes)
    T = y_causal.shape[0]
    if T - D > Wu:
        np.testing.assert_allclose(y_causal[Wu + D:], y_orig[Wu:T - D], rtol=0,
                                   atol=1e-12 * max(1.0, np.abs(y_orig).max()))


@pytest.mark.parametrize("seed", SEEDS[:20])
def test_torch_gradient_reference_forward_on_random_graphs(seed):
    """The torch FP64 causal model (the gradient reference of the
    differentiation form) equals the numpy causal model on the same random
    graphs, noise on."""
    import torch

    from oracle import autodiff as AD

    nodes = random_graph(seed)
    p = W.init_params(nodes, 200 + seed)
    info = M.analyze(nodes)
    x = np.random.default_rng(2000 + seed).standard_normal((info["in_per_step"] * 8, nodes[0]["c_out"]))
    ref = M.run_causal(nodes, p, x, seed=5)
    pt = {i: (torch.tensor(w), None if b is None else torch.tensor(b)) for i, (w, b) in p.items()}
    y = AD.causal_forward(nodes, pt, torch.tensor(x.T.copy()), seed=5).detach().numpy().T
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
