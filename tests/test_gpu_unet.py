"""The warm-start U-Net's CUDA forward and backward (BF16 tensor-core GEMMs, FP32 accumulate)
against the FP64 oracle (oracle/unet.py), through the C ABI.

Tolerances. BF16 keeps 8 significant bits (unit roundoff 2^-9 ~ 2e-3); activations and GEMM
operands are rounded at each of the 15 layers, so the output and the loss stay within ~1e-2.
The parameter gradient is far more sensitive: ReLU units and max-pool winners near a tie switch
under perturbations of that size, which moves whole routes of the backward pass. That
sensitivity is measured on the oracle itself: delta = the oracle's gradient change when only
its weights are rounded to BF16 (3.5 % at c = 8, 7 % at c = 32 on these inputs). The GPU
gradient must stay within 2 delta + 1e-2 of the oracle, point the same way (cosine >= 0.99),
and so must the head's gradient block on its own."""
import numpy as np
import pytest
import torch

import synth
from oracle import unet as ou

pytestmark = pytest.mark.gpu


def _batch(c, B, H, W, seed):
    rng = np.random.default_rng(seed)
    inp = rng.standard_normal((B, 2, H, W)).astype(np.float32)
    inp[:, 1] = np.abs(inp[:, 1])
    tgt = rng.standard_normal((B, H, W)).astype(np.float32)
    return inp, tgt


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


@pytest.mark.parametrize("c,H,W", [(8, 16, 16), (32, 32, 24)])
def test_unet_forward_and_gradient_match_oracle(c, H, W):
    from paper_2609_17636_b300 import UNet
    B = 2
    shapes = synth.unet_layer_shapes(c)
    p = synth.unet_init(c, 3)
    inp, tgt = _batch(c, B, H, W, 4)
    net = UNet(c, max_batch=B, max_hw=H * W)
    net.set_params(p)
    out = net.forward(torch.as_tensor(inp, device="cuda")).cpu().numpy()  # tcgen05 path
    ref = ou.forward(p, shapes, c, inp)
    assert _rel(out, ref) <= 2e-2, _rel(out, ref)
    net.use_tcgen05(False)
    out_mma = net.forward(torch.as_tensor(inp, device="cuda")).cpu().numpy()
    net.use_tcgen05(True)
    assert _rel(out_mma, ref) <= 2e-2, _rel(out_mma, ref)
    # same BF16 operands and FP32 accumulation on both tensor-core paths: only the summation
    # order and the final BF16 rounding of each layer differ
    assert _rel(out, out_mma) <= 1e-2, _rel(out, out_mma)
    loss = net.backward(torch.as_tensor(inp, device="cuda"), torch.as_tensor(tgt, device="cuda"))
    g = net.get_grads()
    lref, gref = ou.loss_and_grad(p, shapes, c, inp, tgt)
    pb = torch.as_tensor(p).to(torch.bfloat16).to(torch.float64).numpy()
    _, gref_b = ou.loss_and_grad(pb, shapes, c, inp, tgt)
    delta = _rel(gref_b, gref)
    assert abs(loss - lref) <= 1e-2 * lref
    assert _rel(g, gref) <= 2 * delta + 1e-2, (_rel(g, gref), delta)
    cos = float(np.dot(g, gref) / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos >= 0.99, cos
    nh = c + 1
    assert _rel(g[-nh:], gref[-nh:]) <= 2 * delta + 1e-2
    net.close()


def test_unet_training_and_inference_sizes_match_oracle():
    """The sizes the network runs at: training batches of 256^2 crops (base width 32, batch 2:
    M = 131072 rows in the first layers' GEMMs, many M tiles and split-K parameter-gradient
    GEMMs) and 512^2 inference (M = 262144). Same tolerances as the small shapes: the output
    and the loss within 2e-2 and 1e-2, the gradient within 2 delta + 1e-2 with delta measured
    on the oracle at this size, cosine >= 0.99."""
    from paper_2609_17636_b300 import UNet
    c, B, H, W = 32, 2, 256, 256
    shapes = synth.unet_layer_shapes(c)
    p = synth.unet_init(c, 9)
    inp, tgt = _batch(c, B, H, W, 10)
    net = UNet(c, max_batch=B, max_hw=512 * 512)
    net.set_params(p)
    x = torch.as_tensor(inp, device="cuda")
    out = net.forward(x).cpu().numpy()
    ref = ou.forward(p, shapes, c, inp)
    assert _rel(out, ref) <= 2e-2, _rel(out, ref)
    loss = net.backward(x, torch.as_tensor(tgt, device="cuda"))
    g = net.get_grads()
    lref, gref = ou.loss_and_grad(p, shapes, c, inp, tgt)
    pb = torch.as_tensor(p).to(torch.bfloat16).to(torch.float64).numpy()
    _, gref_b = ou.loss_and_grad(pb, shapes, c, inp, tgt)
    delta = _rel(gref_b, gref)
    assert abs(loss - lref) <= 1e-2 * lref, (loss, lref)
    assert _rel(g, gref) <= 2 * delta + 1e-2, (_rel(g, gref), delta)
    cos = float(np.dot(g, gref) / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos >= 0.99, cos
    # inference at 512^2 (fully convolutional: the same weights)
    inp1, _ = _batch(c, 1, 512, 512, 11)
    out1 = net.forward(torch.as_tensor(inp1, device="cuda")).cpu().numpy()
    ref1 = ou.forward(p, shapes, c, inp1)
    assert _rel(out1, ref1) <= 2e-2, _rel(out1, ref1)
    net.close()


def test_unet_adam_training_reduces_loss_on_a_fixed_batch():
    from paper_2609_17636_b300 import UNet
    c, B, H, W = 8, 4, 32, 32
    inp, _ = _batch(c, B, H, W, 5)
    tgt = np.maximum(inp[:, 0], 0) * 0.5  # a learnable map of the inputs
    net = UNet(c, max_batch=B, max_hw=H * W)
    net.set_params(synth.unet_init(c, 6))
    x = torch.as_tensor(inp, device="cuda")
    t = torch.as_tensor(tgt, device="cuda")
    first = net.backward(x, t)
    for _ in range(60):
        net.backward(x, t)
        net.adam_step(3e-3)
    last = net.backward(x, t)
    assert last < 0.3 * first, (first, last)
    net.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_warm_start_from_solver_planes(dtype):
    """ivis_unet_warm_start: the network input (s0 dirty, s1 beam weight) is built from the
    solver's planes and the output max(s_out U-Net, 0) is written in their dtype. Against the
    oracle network at the forward test's tolerance, and against ivis_unet_forward on the planes
    ivis_unet_planes scales (the same kernels then: equal to float rounding). The scaling itself
    is one IEEE product per value in the planes' type, so it is compared bit for bit."""
    from paper_2609_17636_b300 import IvisError, UNet, unet_planes
    c, H, W = 8, 32, 40
    shapes = synth.unet_layer_shapes(c)
    p = synth.unet_init(c, 5)
    rng = np.random.default_rng(6)
    npdt = np.float32 if dtype == torch.float32 else np.float64
    dirty = (rng.standard_normal((H, W)) * 3e-4).astype(npdt)
    beam = rng.uniform(0.0, 1.0, (H, W)).astype(npdt)
    s0, s1, s_out = 1.0 / 3e-4, 0.5, 1e-3
    net = UNet(c, max_batch=1, max_hw=H * W)
    net.set_params(p)
    d_t = torch.as_tensor(dirty, device="cuda")
    b_t = torch.as_tensor(beam, device="cuda")
    x0 = net.warm_start(d_t, b_t, s0, s1, s_out)
    assert x0.dtype == dtype and tuple(x0.shape) == (H, W)
    x0 = x0.cpu().numpy()
    planes = unet_planes(d_t, b_t, s0, s1).cpu().numpy()
    want = np.stack([(npdt(s0) * dirty).astype(np.float32), (npdt(s1) * beam).astype(np.float32)])
    assert np.array_equal(planes, want)
    tgt = unet_planes(b_t, None, s1).cpu().numpy()
    assert tgt.shape == (H, W) and np.array_equal(tgt, want[1])
    r = s_out * ou.forward(p, shapes, c, want[None].astype(np.float64))[0]
    assert x0.min() >= 0.0
    # the clamp is 1-Lipschitz, so the forward test's bound carries over unchanged:
    # ||x0 - max(r, 0)|| <= ||s_out out - r|| <= 2e-2 ||r||. (Most outputs of this untrained
    # network are negative: the clamped vector keeps a third of ||r||, so a bound relative to it
    # would be three times tighter than the forward's.)
    err = float(np.linalg.norm(x0 - np.maximum(r, 0.0)))
    assert err <= 2e-2 * np.linalg.norm(r), err / np.linalg.norm(r)
    out = net.forward(torch.as_tensor(want[None], device="cuda")).cpu().numpy()[0]
    via_forward = np.maximum(npdt(s_out) * out.astype(npdt), 0.0)
    assert _rel(x0, via_forward) <= 1e-6, _rel(x0, via_forward)
    with pytest.raises(IvisError):  # W not a multiple of 8
        net.warm_start(d_t[:, :36].contiguous(), b_t[:, :36].contiguous(), s0, s1, s_out)
    with pytest.raises(ValueError):
        net.warm_start(d_t, b_t.float() if dtype == torch.float64 else b_t.double(), s0, s1, s_out)
    net.close()
