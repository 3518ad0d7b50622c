"""Pins for the oracle's convolutions (Eq. 1, section 2.1) against brute force,
an independent library routine (torch CPU float64) and closed forms."""
import numpy as np
import pytest
import torch

from oracle import conv as C


@pytest.mark.parametrize("stride,dilation,k,pl,pr", [
    (1, 1, 3, 1, 1), (1, 2, 3, 2, 2), (1, 3, 5, 6, 6), (2, 1, 5, 2, 2),
    (3, 1, 7, 3, 3), (4, 1, 9, 4, 4), (2, 2, 3, 1, 3), (1, 1, 4, 2, 1), (1, 1, 1, 0, 0),
])
def test_correlate_matches_quadruple_loop(stride, dilation, k, pl, pr):
    rng = np.random.default_rng(10 + k + stride)
    x = rng.standard_normal((3, 29))
    w = rng.standard_normal((4, 3, k))
    xp = C.zero_pad(x, pl, pr)
    np.testing.assert_allclose(C.correlate(xp, w, stride, dilation),
                               C.correlate_loops(xp, w, stride, dilation), rtol=0, atol=1e-12)


@pytest.mark.parametrize("stride,dilation,k,pad", [(1, 1, 3, 1), (1, 9, 3, 9), (4, 1, 9, 4),
                                                   (16, 1, 64, 24), (2, 1, 5, 2), (1, 1, 7, 3)])
def test_conv1d_matches_torch(stride, dilation, k, pad):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 160))
    w = rng.standard_normal((6, 5, k))
    b = rng.standard_normal(6)
    ref = torch.nn.functional.conv1d(torch.from_numpy(x)[None], torch.from_numpy(w),
                                     torch.from_numpy(b), stride=stride, padding=pad,
                                     dilation=dilation)[0].numpy()
    out = C.conv1d(x, w, b, stride, dilation, pad, pad)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-11)


def test_conv1d_asymmetric_padding_matches_torch_after_manual_pad():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 40))
    w = rng.standard_normal((3, 2, 4))
    ref = torch.nn.functional.conv1d(
        torch.nn.functional.pad(torch.from_numpy(x)[None], (3, 0)), torch.from_numpy(w))[0].numpy()
    np.testing.assert_allclose(C.conv1d(x, w, None, 1, 1, 3, 0), ref, atol=1e-12)


@pytest.mark.parametrize("stride,k", [(4, 8), (2, 4), (16, 64), (3, 3), (2, 5)])
def test_conv_transpose_matches_loops_and_torch(stride, k):
    rng = np.random.default_rng(3 + k)
    x = rng.standard_normal((4, 11))
    w = rng.standard_normal((4, 3, k))
    full = C.conv_transpose_full(x, w, stride)
    np.testing.assert_allclose(full, C.conv_transpose_full_loops(x, w, stride), atol=1e-12)
    ref = torch.nn.functional.conv_transpose1d(torch.from_numpy(x)[None], torch.from_numpy(w),
                                               stride=stride)[0].numpy()
    np.testing.assert_allclose(full, ref, atol=1e-11)


def test_conv_transpose_box_kernel_is_nearest_neighbour_upsampling():
    # w[c][c][p:p+S] = 1 -> after cropping p: out[t] = x[floor(t / S)]
    s, p = 4, 2
    x = np.arange(1.0, 8.0)[None, :]
    w = np.zeros((1, 1, 2 * s))
    w[0, 0, p:p + s] = 1.0
    out = C.conv_transpose_full(x, w, s)[:, p:p + x.shape[1] * s]
    np.testing.assert_array_equal(out[0], np.repeat(x[0], s))


def test_delta_kernel_is_a_shift():
    x = np.random.default_rng(4).standard_normal((1, 30))
    w = np.zeros((1, 1, 5))
    w[0, 0, 3] = 1.0
    # valid correlation with a delta at tap 3 reads x[i + 3]
    np.testing.assert_array_equal(C.correlate(x, w)[0], x[0, 3:3 + 26])


def test_leaky_relu():
    x = np.array([-5.0, -0.5, 0.0, 0.5, 3.0])
    np.testing.assert_array_equal(C.leaky_relu(x), [-1.0, -0.1, 0.0, 0.5, 3.0])
