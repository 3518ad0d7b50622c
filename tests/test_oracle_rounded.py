"""Pins for the oracle's rounded-operand gradients (oracle/autodiff.py,
``rounded=``): the reference for differentiating a BF16/FP16 forward.  The
rounding is checked against its bit-level definition (BF16: the upper half of
the float32 word, rounded to nearest even) and numpy's float16 cast; the
gradients of one- and two-layer models against closed forms written here with
numpy, including a case where rounding moves a LeakyReLU input across zero
(the gradient must take the derivative on the rounded forward's side)."""
import numpy as np
import pytest
import torch

from oracle import autodiff as AD
from oracle import model as M
from paper_2204_07064_gb300 import workloads as W


def _bf16_rne(v):
    """float64 -> float32 -> bfloat16 by the bit rule: add 0x7FFF plus the
    kept word's lowest bit, then clear the low 16 bits."""
    u = np.asarray(v, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_round_to_matches_bit_definitions():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        # exact ties for both formats: 1 + half an ulp, 1 + 1.5 ulp
                        [1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 2.0 ** -8)]])
    got = AD.round_to(torch.tensor(v), "bf16").numpy()
    np.testing.assert_array_equal(got, _bf16_rne(v))
    v = v[np.abs(v) < 6e4]  # inside float16's range
    got = AD.round_to(torch.tensor(v), "f16").numpy()
    np.testing.assert_array_equal(got, v.astype(np.float32).astype(np.float16).astype(np.float64))
    # ties go to the even neighbour
    assert AD.round_to(torch.tensor([1 + 2.0 ** -8]), "bf16").item() == 1.0
    assert AD.round_to(torch.tensor([1 + 3 * 2.0 ** -8]), "bf16").item() == 1 + 2.0 ** -6


def _f16(v):
    return np.asarray(v, np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


def _row_rounded(w2, rq):
    """Rows of a [rows][cols] matrix scaled to max |w| = 1 in float32, rounded
    by rq, scaled back."""
    w32 = np.asarray(w2, np.float64).astype(np.float32)
    sc = np.abs(w32).max(axis=1, keepdims=True)
    sc = np.where(sc > 0, sc, np.float32(1))
    return rq((w32 / sc).astype(np.float64)) * sc.astype(np.float64)


def _one_by_one(nodes_acts, cin=3, cout=2):
    nodes = [W.input_node(cin)]
    c = cin
    for a in nodes_acts:
        nodes.append(W._node("conv", [len(nodes) - 1], c, cout, k=1, act_in=a))
        c = cout
    return nodes


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("act", [None, "leaky"])
def test_rounded_single_layer_closed_form(fmt, act):
    """y = Wq act(x)q + b, L = sum(r * y): dL/dx = (Wq^T r) act'(x),
    dL/dW = r act(x)q^T, dL/db = sum over time of r; Wq rounded row by row
    after scaling each output channel's row to max |w| = 1."""
    nodes = _one_by_one([act])
    p = W.init_params(nodes, 4)
    x = W.signal(5, 7, 3)
    r = np.random.default_rng(6).standard_normal((7, 2))
    rq = _bf16_rne if fmt == "bf16" else _f16
    w, b = p[1]
    wq = _row_rounded(w[:, :, 0], rq)
    assert np.abs(wq - rq(w[:, :, 0])).max() > 0  # the row scale matters
    a = np.where(x >= 0, x, 0.2 * x) if act else x
    d = np.where(x > 0, 1.0, 0.2) if act else np.ones_like(x)
    loss, gx, gw = AD.gradients(nodes, p, x, r, rounded={1: fmt})
    np.testing.assert_allclose(loss, np.sum(r * (rq(a) @ wq.T + b)), rtol=1e-12)
    np.testing.assert_allclose(gx, (r @ wq) * d, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gw[1][0][:, :, 0], r.T @ rq(a), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gw[1][1], r.sum(0), rtol=1e-12)


def test_rounded_kink_takes_the_rounded_side():
    """Two 1x1 layers, LeakyReLU between them.  With x = (1 + 3*2^-9,
    1 + 2^-7 + 2^-10) the exact first output is x0 - x1 + 2^-12 < 0, but both
    inputs round to 1 + 2^-7 in BF16, so the rounded layer outputs +2^-12 and
    the second layer's LeakyReLU passes the gradient with slope 1, not 0.2."""
    nodes = [W.input_node(2), W._node("conv", [0], 2, 1, k=1), W._node("conv", [1], 1, 1, k=1, act_in="leaky")]
    p = {1: (np.array([[[1.0], [-1.0]]]), np.array([2.0 ** -12])), 2: (np.array([[[2.0]]]), np.array([0.0]))}
    x = np.array([[1 + 3 * 2.0 ** -9, 1 + 2.0 ** -7 + 2.0 ** -10]])
    r = np.array([[1.0]])
    y1 = x[0, 0] - x[0, 1] + 2.0 ** -12
    assert y1 < 0
    _, gx, _ = AD.gradients(nodes, p, x, r)
    np.testing.assert_allclose(gx, [[0.2 * 2.0, -0.2 * 2.0]], rtol=1e-12)
    _, gx, gw = AD.gradients(nodes, p, x, r, rounded={1: "bf16", 2: "bf16"})
    np.testing.assert_allclose(gx, [[2.0, -2.0]], rtol=1e-12)
    # dL/dW1 = (W2 * slope * r) * round(x) = 2 * (1 + 2^-7) per input
    np.testing.assert_allclose(gw[1][0][0, :, 0], [2 * (1 + 2.0 ** -7)] * 2, rtol=1e-12)
    np.testing.assert_allclose(gw[2][0][0, 0, 0], 2.0 ** -12, rtol=1e-12)


def test_rounding_representable_operands_changes_nothing():
    """Weights and inputs on a coarse dyadic grid, every weight row's largest
    magnitude 1/2 (so the row scale is a power of two), are BF16 numbers
    already: the rounded model is then the exact one, gradients included."""
    nodes = W.tiny_stack()
    p = W.init_params(nodes, 1)

    def grid(w):
        w = np.clip(np.round(w * 16) / 16, -0.5, 0.5)
        w[:, 0, 0] = 0.5
        return w
    p = {i: (grid(w), None if b is None else np.round(b * 16) / 16) for i, (w, b) in p.items()}
    x = np.round(W.signal(3, 40, 16) * 8) / 8
    y = M.run_causal(nodes, p, x, seed=3)
    r = np.random.default_rng(1).standard_normal(y.shape)
    convs = {i: "bf16" for i, nd in enumerate(nodes) if nd["op"] in ("conv", "convt")}
    l0, gx0, gw0 = AD.gradients(nodes, p, x, r, seed=3)
    l1, gx1, gw1 = AD.gradients(nodes, p, x, r, seed=3, rounded=convs)
    # only the first layer's input is on the grid; deeper activations are not,
    # so compare the first layer alone on a one-layer model as well
    one = nodes[:2]
    y1 = M.run_causal(one, {1: p[1]}, x, seed=3)
    r1 = np.random.default_rng(2).standard_normal(y1.shape)
    a = AD.gradients(one, {1: p[1]}, x, r1, seed=3)
    b = AD.gradients(one, {1: p[1]}, x, r1, seed=3, rounded={1: "bf16"})
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2][1][0], b[2][1][0])
    # the deep model differs, but only by rounding-sized amounts
    assert abs(l1 - l0) <= 2.0 ** -6 * np.sum(np.abs(r * y))
    assert np.linalg.norm(gx1 - gx0) <= 0.1 * np.linalg.norm(gx0)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_round_weights_row_groups(fmt):
    """A conv's row is an output channel; a transposed conv's row is an
    (output channel, output phase) pair.  Scaling one row by a factor leaves
    every other row's rounded weights unchanged, and a row whose largest
    magnitude is already 1 is rounded plainly."""
    rng = np.random.default_rng(3)
    rq = _bf16_rne if fmt == "bf16" else _f16
    w = rng.standard_normal((5, 4, 3))  # conv [cout][cin][k]
    q = AD.round_weights(torch.tensor(w), fmt, "conv").numpy()
    np.testing.assert_array_equal(q, _row_rounded(w.reshape(5, 12), rq).reshape(5, 4, 3))
    w1 = w.copy()
    w1[2] *= 3.3
    q1 = AD.round_weights(torch.tensor(w1), fmt, "conv").numpy()
    np.testing.assert_array_equal(np.delete(q1, 2, axis=0), np.delete(q, 2, axis=0))
    S, K = 2, 4
    wt = rng.standard_normal((4, 3, K))  # convT [cin][cout][k], phase of tap k = k % S
    qt = AD.round_weights(torch.tensor(wt), fmt, "convt", S).numpy()
    for ph in range(S):
        for o in range(3):
            row = wt[:, o, ph::S].reshape(1, -1)
            np.testing.assert_array_equal(qt[:, o, ph::S].reshape(1, -1), _row_rounded(row, rq))
    wt1 = wt.copy()
    wt1[:, 1, 1::S] *= 3.3  # output channel 1, phase 1 only
    qt1 = AD.round_weights(torch.tensor(wt1), fmt, "convt", S).numpy()
    keep = np.ones_like(qt, bool)
    keep[:, 1, 1::S] = False
    np.testing.assert_array_equal(qt1[keep], qt[keep])
    # rows with max |w| = 1: plain rounding
    u = w / np.abs(w).max(axis=(1, 2), keepdims=True)
    np.testing.assert_array_equal(AD.round_weights(torch.tensor(u), fmt, "conv").numpy(), rq(u))
