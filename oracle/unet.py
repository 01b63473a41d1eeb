"""FP64 CPU oracle of the warm-start U-Net (test infrastructure only).

Plain PyTorch CPU operations in float64: 'same' 3x3 cross-correlation with zero padding,
ReLU, 2x2 max pooling, nearest-neighbour 2x upsampling, channel concatenation, a 1x1 head and
the mean-squared-error loss; the gradient is PyTorch's reverse-mode differentiation of that
forward pass. The parameter layout is the library's flat vector (per layer W[cout][3 dy + dx][cin]
then bias[cout]; head weights then bias). Pinned by tests/test_oracle_unet.py (scipy
correlation, finite differences).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

__all__ = ["unpack", "forward", "loss_and_grad"]


def unpack(params: np.ndarray, shapes, c: int):
    """Per-layer (weight [cout][cin][3][3], bias) tensors and the head from the flat vector."""
    return _unpack_t(torch.as_tensor(np.asarray(params, dtype=np.float64)), shapes, c)


def _net(layers, hw, hb, x):
    relu = torch.relu
    conv = lambda t, wb: relu(F.conv2d(t, wb[0], wb[1], padding=1))
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    a0 = conv(x, layers[0]); a1 = conv(a0, layers[1])
    a2 = conv(F.max_pool2d(a1, 2), layers[2]); a3 = conv(a2, layers[3])
    a4 = conv(F.max_pool2d(a3, 2), layers[4]); a5 = conv(a4, layers[5])
    a6 = conv(F.max_pool2d(a5, 2), layers[6]); a7 = conv(a6, layers[7])
    a8 = conv(torch.cat([up(a7), a5], 1), layers[8]); a9 = conv(a8, layers[9])
    a10 = conv(torch.cat([up(a9), a3], 1), layers[10]); a11 = conv(a10, layers[11])
    a12 = conv(torch.cat([up(a11), a1], 1), layers[12]); a13 = conv(a12, layers[13])
    return torch.einsum("bchw,c->bhw", a13, hw) + hb


def forward(params, shapes, c, inp):
    """inp float [B][2][H][W] -> output [B][H][W] (float64 numpy)."""
    layers, hw, hb = unpack(params, shapes, c)
    with torch.no_grad():
        return _net(layers, hw, hb, torch.as_tensor(np.asarray(inp, dtype=np.float64))).numpy()


def loss_and_grad(params, shapes, c, inp, tgt):
    """Mean squared error against tgt [B][H][W] and its gradient w.r.t. the flat parameters."""
    p = torch.as_tensor(np.asarray(params, dtype=np.float64)).clone().requires_grad_(True)
    layers, hw, hb = _unpack_t(p, shapes, c)
    out = _net(layers, hw, hb, torch.as_tensor(np.asarray(inp, dtype=np.float64)))
    loss = torch.mean((out - torch.as_tensor(np.asarray(tgt, dtype=np.float64))) ** 2)
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()


def _unpack_t(p, shapes, c):
    out, off = [], 0
    for (ca, _, cb, co, _) in shapes:
        cin = ca + cb
        w = p[off:off + co * 9 * cin].reshape(co, 3, 3, cin).permute(0, 3, 1, 2)
        off += co * 9 * cin
        b = p[off:off + co]
        off += co
        out.append((w, b))
    return out, p[off:off + c], p[off + c:off + c + 1]
