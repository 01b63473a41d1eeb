"""The allocation-free single-dish prediction (ivis_sd_predict_noalloc) against the plan-based
ivis_sd_predict, through the C ABI.

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
    for trial in range(2):
        sky = torch.as_tensor(rng.uniform(0, 1, (nchan, n, n)), dtype=torch.float32, device="cuda")
        ref = plan.sd_predict(sky)
        out = torch.full_like(sky, float("nan"))
        assert _noalloc(L, sky, n, nchan, fwhm, out) == 0, L.ivis_last_error(None)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(out.double() - ref.double()) /
                    torch.linalg.vector_norm(ref.double()))
        assert err <= TOL, (trial, err)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2609_17636_b300 import load
    L = load()
    sky = torch.zeros(1025 * 1025, device="cuda")
    out = torch.zeros_like(sky)
    assert _noalloc(L, sky, 1025, 1, 4.0, out) == 1
    assert b"too large" in L.ivis_last_error(None)
    small = torch.zeros(64 * 64, device="cuda")
    assert _noalloc(L, small, 64, 1, 2000.0, torch.zeros_like(small)) == 1
    assert b"too wide" in L.ivis_last_error(None)
