"""Pins of the FP64 U-Net oracle: its convolution against scipy's correlation, its gradient
against central finite differences, and its parameter count and layout."""
import numpy as np
import scipy.signal
import torch
import torch.nn.functional as F

import synth
from oracle import unet as ou


def test_parameter_count_matches_layer_shapes():
    c = 32
    shapes = synth.unet_layer_shapes(c)
    n = synth.unet_num_params(c)
    p = synth.unet_init(c, 0)
    assert p.shape == (n,) and n == 1_946_593  # summed by hand over the 14 layers + head
    layers, hw, hb = ou.unpack(p, shapes, c)
    assert len(layers) == 14 and hw.shape == (c,) and hb.shape == (1,)


def test_layer_is_same_cross_correlation_with_zero_padding():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 3, 9, 11))
    w = rng.standard_normal((2, 3, 3, 3))
    got = F.conv2d(torch.as_tensor(x), torch.as_tensor(w), padding=1).numpy()
    for co in range(2):
        ref = sum(scipy.signal.correlate2d(x[0, ci], w[co, ci], mode="same", boundary="fill")
                  for ci in range(3))
        assert np.allclose(got[0, co], ref, atol=1e-12)


def test_flat_layout_tap_order():
    """W[cout][3 dy + dx][cin] in the flat vector maps to weight[co][ci][dy][dx]."""
    c = 8
    shapes = synth.unet_layer_shapes(c)
    p = np.zeros(synth.unet_num_params(c))
    # layer 0: cin = 2; set W[co=3][tap=5 (dy=1,dx=2)][ci=1]
    p[3 * 18 + 5 * 2 + 1] = 7.0
    layers, _, _ = ou.unpack(p, shapes, c)
    assert layers[0][0][3, 1, 1, 2] == 7.0 and float(layers[0][0].abs().sum()) == 7.0


def test_gradient_central_differences_tiny_net():
    c = 8
    shapes = synth.unet_layer_shapes(c)
    p = synth.unet_init(c, 1).astype(np.float64)
    rng = np.random.default_rng(2)
    inp = rng.standard_normal((2, 2, 8, 8))
    tgt = rng.standard_normal((2, 8, 8))
    _, g = ou.loss_and_grad(p, shapes, c, inp, tgt)
    h = 1e-6
    for i in rng.choice(p.size, 25, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = ou.loss_and_grad(p + e, shapes, c, inp, tgt)
        lm, _ = ou.loss_and_grad(p - e, shapes, c, inp, tgt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()) + 1e-4 * abs(g[i]), (i, fd, g[i])


def _offsets(shapes):
    """(weight offset, bias offset) of each 3x3 layer in the flat vector, and the head's."""
    offs, off = [], 0
    for (ca, _, cb, co, _) in shapes:
        offs.append((off, off + co * 9 * (ca + cb)))
        off += co * 9 * (ca + cb) + co
    return offs, off


def test_decoder_concatenation_order_by_hand():
    """Decoder 'a' layers read the upsampled deeper tensor's channels first, then the skip
    channels. Hand-built weights: every layer outputs the constant relu(bias) = its index + 1,
    except that from decoder layer L on channel 0 is passed through the centre tap alone. The
    output is then the deeper tensor's constant (L) -- the skip tensor's would differ."""
    c = 8
    shapes = synth.unet_layer_shapes(c)
    offs, head = _offsets(shapes)
    for L in (8, 10, 12):
        p = np.zeros(synth.unet_num_params(c))
        for i, (ca, _, cb, co, _) in enumerate(shapes):
            w_off, b_off = offs[i]
            if i < L:
                p[b_off:b_off + co] = i + 1
            else:  # W[co=0][tap=4 (dy=1, dx=1)][ci=0] = 1, zero bias
                p[w_off + 0 * 9 * (ca + cb) + 4 * (ca + cb) + 0] = 1.0
        p[head] = 1.0  # head weight of channel 0; head bias 0
        out = ou.forward(p, shapes, c, np.zeros((1, 2, 16, 16)))
        assert np.all(out == float(L)), (L, np.unique(out))


def test_pooling_is_max_and_upsampling_is_nearest_by_hand():
    """Hand-built weights that pass input plane 0 through channel 0 of every layer (centre tap
    1, zero bias) make the network the composition of its resampling steps: three 2x2 max
    poolings down and three nearest 2x upsamplings back, i.e. the maximum of each 8x8 block
    repeated over the block (the input is non-negative, so the ReLUs pass it unchanged)."""
    c = 8
    shapes = synth.unet_layer_shapes(c)
    offs, head = _offsets(shapes)
    p = np.zeros(synth.unet_num_params(c))
    for i, (ca, _, cb, co, _) in enumerate(shapes):
        p[offs[i][0] + 4 * (ca + cb)] = 1.0  # W[0][tap 4][ci 0]
    p[head] = 1.0
    rng = np.random.default_rng(5)
    inp = np.zeros((1, 2, 16, 24))
    inp[0, 0] = rng.uniform(0.0, 1.0, (16, 24))
    inp[0, 1] = rng.standard_normal((16, 24))  # plane 1 is not routed anywhere
    out = ou.forward(p, shapes, c, inp)[0]
    block = inp[0, 0].reshape(2, 8, 3, 8).max(axis=(1, 3))
    assert np.array_equal(out, np.kron(block, np.ones((8, 8))))
