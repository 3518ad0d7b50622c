"""Pins for the oracle's causal reconfiguration (section 3): Eq. 2, Eq. 3, the
cumulated lag, and pure-delay behaviour of identity networks."""
import numpy as np
import pytest

from oracle import model as M
from paper_2204_07064_gb300 import workloads as W


def test_eq2_alignment_invariants():
    for s in range(1, 9):
        for r in range(0, 12):
            for dc in range(0, 40):
                da = M.stride_alignment(s, r, dc)
                assert 0 <= da < s
                assert (dc + r + da) % s == 0
                # minimal: no smaller non-negative extra delay aligns the lag
                assert all((dc + r + e) % s for e in range(da))


def test_worked_delays():
    """Delays re-derived by hand from section 3's rules (stride-1 conv adds R;
    ConvT maps D to D*S + crop; strided conv (D + R + Da)/S; merges take the max)."""
    assert M.analyze(W.tiny_stack())["delay"] == 1 + 2 + 4
    # decoder: pre 1; each stage D -> D*r + r/2 then + (1+3+9); heads + 3;
    # inverse PQMF D*16 + 24
    d = 1
    for r in (4, 4, 4, 2):
        d = d * r + r // 2 + 13
    d = (d + 3) * 16 + 24
    dec = W.rave_decoder()
    info = M.analyze(dec)
    assert info["delay"] == d == 12424
    heads = [i for i, n in enumerate(dec) if n["op"] == "heads"][0]
    assert info["A"][heads] == [0, 2, 1]
    enc = W.rave_encoder()
    ie = M.analyze(enc)
    assert ie["delay"] == 3
    assert [ie["Da"][i] for i, n in enumerate(enc) if n["op"] == "conv" and n["stride"] > 1] == [8, 3, 1, 2, 0]
    assert ie["in_per_step"] == 2048


def test_merge_inputs_aligned():
    dec = W.rave_decoder()
    info = M.analyze(dec)
    for i, n in enumerate(dec):
        if n["op"] in ("add", "heads"):
            delays = {info["D"][u] + a for u, a in zip(n["inputs"], info["A"][i])}
            assert len(delays) == 1


def test_cache_size_closed_form():
    """Cache = sum over tensors of (frames kept) x channels.  Decoder, by hand:
    latent 2*128, pre 1*1024, per stage (C = 512, 256, 128, 64): ConvT output
    keeps 2 (conv d=1 and skip 1), unit outputs keep 6 and 18 (next dilated
    conv), last unit keeps 1 (next ConvT) except in the last stage where it
    feeds the heads (7-tap conv: 6); heads: noise1 2*16, amp 2*16 and noise2 1*16
    (Eq. 3 delays), combined output 3*16 (inverse PQMF, 4 taps per phase)."""
    dec = W.rave_decoder()
    info = M.analyze(dec)
    expect = 2 * 128 + 1024
    for c in (512, 256, 128):
        expect += (2 + 6 + 18 + 1) * c
    expect += (2 + 6 + 18 + 6) * 64
    expect += 2 * 16 + 2 * 16 + 1 * 16 + 3 * 16
    assert M.cache_elements(dec, info) == expect == 27648
    tiny = W.tiny_stack()
    assert M.cache_elements(tiny, M.analyze(tiny)) == (2 + 4 + 8) * 16


def _identity_model(nodes):
    nodes = W.strip_activations(nodes)
    return nodes, W.identity_params(nodes)


def test_identity_tiny_is_pure_delay():
    nodes, p = _identity_model(W.tiny_stack())
    x = W.signal(3, 300, 16)
    d = M.analyze(nodes)["delay"]
    np.testing.assert_array_equal(M.run_original(nodes, p, x), x)
    yc = M.run_causal(nodes, p, x)
    np.testing.assert_array_equal(yc[d:], x[:-d])
    np.testing.assert_array_equal(yc[:d], 0.0)


def test_identity_encoder_is_delayed_decimation():
    """Identity weights make the encoder a decimator by 2048 of input channel 0;
    the causal model must be that decimation delayed by 3 latent frames.  Without
    Eq. 2's extra delays it would sample the input at the wrong phase."""
    nodes, p = _identity_model(W.rave_encoder())
    x = W.signal(4, 2048 * 12, 1)
    yo = M.run_original(nodes, p, x)
    np.testing.assert_array_equal(yo[:, 0], x[::2048, 0])
    d = M.analyze(nodes)["delay"]
    yc = M.run_causal(nodes, p, x)
    np.testing.assert_array_equal(yc[d:, 0], yo[:-d, 0])
    np.testing.assert_array_equal(yc[:d], 0.0)


def test_identity_decoder_trunk_is_delayed_upsampling():
    """Decoder trunk (no heads / PQMF) with identity weights: each residual unit
    adds an identity branch to its skip (x -> 2x), each ConvT repeats frames.
    The causal output must equal that, delayed by the computed D; a wrong
    branch delay (Eq. 3) would mix misaligned frames."""
    dec = W.rave_decoder()
    trunk = [n for n in dec if n["name"] not in ("wave", "amp", "noise1", "noise2", "heads", "ipqmf")]
    nodes, p = _identity_model(trunk)
    x = W.signal(5, 12, 128)
    yo = M.run_original(nodes, p, x)
    up = np.repeat(x[:, :64], 128, axis=0) * 2.0 ** 12
    np.testing.assert_array_equal(yo, up)
    d = M.analyze(nodes)["delay"]
    assert d == (12424 - 24) // 16 - 3
    yc = M.run_causal(nodes, p, x)
    np.testing.assert_array_equal(yc[d:], yo[:-d])
    np.testing.assert_array_equal(yc[:d], 0.0)


def test_identity_parallel_branches_with_unequal_delays():
    """Two branches of different delay (k=7 pad 3/3 vs k=3 pad 1/1, and a
    strided branch pair) merged by an add: Eq. 3 must re-synchronise them."""
    n = [W.input_node(2)]
    n.append(W._node("conv", [0], 2, 2, k=7, pad_left=3, pad_right=3, name="a"))
    n.append(W._node("conv", [0], 2, 2, k=3, pad_left=1, pad_right=1, name="b"))
    n.append(W._node("conv", [2], 2, 2, k=5, pad_left=0, pad_right=4, name="c"))
    n.append(W._node("add", [1, 3], 2, 2, bias=False))
    n.append(W._node("conv", [4], 2, 2, k=5, stride=2, pad_left=2, pad_right=2, name="s"))
    n.append(W._node("conv", [4], 2, 2, k=3, stride=2, pad_left=1, pad_right=1, name="t"))
    n.append(W._node("add", [5, 6], 2, 2, bias=False))
    nodes, p = _identity_model(n)
    info = M.analyze(nodes)
    assert info["A"][4] == [2, 0] and info["D"][4] == 5
    x = W.signal(6, 64, 2)
    yo = M.run_original(nodes, p, x)
    np.testing.assert_array_equal(yo, 4.0 * x[::2])
    yc = M.run_causal(nodes, p, x)
    d = info["delay"]
    np.testing.assert_array_equal(yc[d:], yo[:-d])


def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle (on the CPU) and check that the
    identity-network pins above detect them."""
    nodes, p = _identity_model(W.rave_encoder())
    x = W.signal(4, 2048 * 12, 1)
    yo = M.run_original(nodes, p, x)

    def encoder_pin():
        d = M.analyze(nodes)["delay"]
        yc = M.run_causal(nodes, p, x)
        return np.array_equal(yc[d:, 0], yo[:-d, 0])

    assert encoder_pin()
    # (1) Eq. 2 dropped: no extra delay before strided layers
    monkeypatch.setattr(M, "stride_alignment", lambda s, r, dc: 0)
    with pytest.raises(AssertionError):
        M.analyze(nodes)  # the lag is then not a multiple of the stride
    # (2) Eq. 2 with the remainder subtracted the wrong way round
    monkeypatch.setattr(M, "stride_alignment", lambda s, r, dc: (r + dc) % s)
    try:
        ok = encoder_pin()
    except AssertionError:
        ok = False
    assert not ok
    monkeypatch.undo()
    # (3) Eq. 3 dropped: merged branches not delayed
    monkeypatch.setattr(M, "_delay", lambda v, a: v)
    trunk = [nd for nd in W.rave_decoder()
             if nd["name"] not in ("wave", "amp", "noise1", "noise2", "heads", "ipqmf")]
    tn, tp = _identity_model(trunk)
    z = W.signal(5, 12, 128)
    d = M.analyze(tn)["delay"]
    yc = M.run_causal(tn, tp, z)
    yo2 = M.run_original(tn, tp, z)
    assert len(yc) > d
    assert not np.array_equal(yc[d:], yo2[:-d])
