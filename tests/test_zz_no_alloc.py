"""The allocation-free single-dish prediction (ivis_sd_predict_noalloc) against the plan-based
ivis_sd_predict and the FP64 oracle's dish convolution, through the C ABI.

Callers that cannot allocate device memory when they need the dish-beam model (inside a
region whose memory a pool or another framework owns, or a host that forbids allocation after
start-up) use the no-alloc entry point; its scratch is a fixed device array inside the
library. Two calls in a row must both agree with the plan-based result (the array keeps the
previous call's contents, which must not leak into the next result). This file is collected
last so that a run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the FP32 path's tolerance


def _noalloc(L, sky, n, nchan, fwhm, out):
    return L.ivis_sd_predict_noalloc(ctypes.c_void_p(sky.data_ptr()), n, nchan, float(fwhm),
                                     ctypes.c_void_p(out.data_ptr()), None)


def test_noalloc_sd_predict_matches_plan_path_twice():
    from paper_2609_17636_b300 import Plan, load
    L = load()
    rng = np.random.default_rng(11)
    n, nchan, fwhm = 256, 2, 13.7
    plan = Plan(n, nchan, 1, 16, 1e-5, "fp32", lambda_s=1.0)
    plan.set_pointing(0, n // 2, n // 2, torch.ones(16, 16, device="cuda"))
    for c in range(nchan):
        plan.set_vis(0, c, torch.zeros((0, 3), device="cuda"), None, None)
        plan.set_sd(c, torch.zeros(n, n, device="cuda"), 1.0, fwhm)
    b = oracle.dish_kernel(fwhm)
    for trial in range(2):
        sky = torch.as_tensor(rng.uniform(0, 1, (nchan, n, n)), dtype=torch.float32, device="cuda")
        ref = plan.sd_predict(sky)
        out = torch.full_like(sky, float("nan"))
        assert _noalloc(L, sky, n, nchan, fwhm, out) == 0, L.ivis_last_error(None)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(out.double() - ref.double()) /
                    torch.linalg.vector_norm(ref.double()))
        assert err <= TOL, (trial, err)
        o = out.double().cpu().numpy()
        want = np.stack([oracle.dish_conv(sky[c].double().cpu().numpy(), b) for c in range(nchan)])
        assert np.linalg.norm(o - want) <= TOL * np.linalg.norm(want), trial
    plan.close()


def test_noalloc_widest_beam_matches_oracle():
    """The widest beam the scratch takes: ceil(4 sigma) = 812 (1625 taps) on a 64^2 image, so
    every output sums taps that run far past the image on both sides."""
    from paper_2609_17636_b300 import load
    L = load()
    n, fwhm = 64, 477.8
    b = oracle.dish_kernel(fwhm)
    assert b.shape[0] == 2 * 812 + 1
    sky = torch.as_tensor(np.random.default_rng(12).uniform(0, 1, (1, n, n)), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(sky)
    assert _noalloc(L, sky, n, 1, fwhm, out) == 0, L.ivis_last_error(None)
    torch.cuda.synchronize()
    want = oracle.dish_conv(sky[0].double().cpu().numpy(), b)
    assert np.linalg.norm(out[0].double().cpu().numpy() - want) <= TOL * np.linalg.norm(want)


def test_noalloc_refuses_a_capturing_stream():
    """The call copies its taps from host memory and waits for the stream, so on a stream that
    is being captured it returns IVIS_ERR_STATE and leaves the capture intact."""
    from paper_2609_17636_b300 import load
    L = load()
    sky = torch.zeros(1, 32, 32, device="cuda")
    out = torch.zeros_like(sky)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        sky.add_(1.0)
        st = L.ivis_sd_predict_noalloc(ctypes.c_void_p(sky.data_ptr()), 32, 1, 3.0,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
        g.capture_end()
    assert st == 2 and b"capturing" in L.ivis_last_error(None)
    g.replay()
    torch.cuda.synchronize()
    assert float(sky.min()) == 1.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2609_17636_b300 import load
    L = load()
    sky = torch.zeros(1025 * 1025, device="cuda")
    out = torch.zeros_like(sky)
    assert _noalloc(L, sky, 1025, 1, 4.0, out) == 1
    assert b"too large" in L.ivis_last_error(None)
    small = torch.zeros(64 * 64, device="cuda")
    for fwhm in (478.5, 900.0, 2000.0):  # ceil(4 sigma) = 813, 1529, 3398
        assert _noalloc(L, small, 64, 1, fwhm, torch.zeros_like(small)) == 1
        assert b"too wide" in L.ivis_last_error(None)
