"""Feathering (the paper's short-spacing appendix) through ivis_feather against the oracle's
numpy restatement, relative L2 1e-9 (FP64) and 1e-5 (FP32)."""

import numpy as np
import pytest
import torch

import oracle
import synth
from _data import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,nchan", [(16, 1), (128, 3), (512, 2)])
def test_feather_matches_oracle(precision, n, nchan):
    from paper_2609_17636_b300 import Plan
    cell = 7.0 * synth.ARCSEC
    plan = Plan(n, nchan, 1, 16, cell, precision)
    rng = np.random.default_rng(n + nchan)
    i_int = np.stack([synth.lognormal_sky(rng, n) for _ in range(nchan)])
    i_sd = np.stack([synth.lognormal_sky(rng, n, i0=2e-3) for _ in range(nchan)]).astype(np.float32)
    theta = 30.0 * 60.0 * synth.ARCSEC if n >= 256 else 40.0 * cell
    scale = oracle.rayleigh_jeans_factor(synth.HI_FREQ_HZ) * 1e3
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = plan.feather(torch.as_tensor(i_int, dtype=dt, device="cuda"),
                       torch.as_tensor(i_sd, device="cuda"), theta, scale)
    ref = oracle.feather(i_int.astype(np.float64) if precision == "fp64" else i_int.astype(np.float32),
                         i_sd, theta / cell, scale)
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert rel_l2(out.cpu().numpy(), ref) <= tol, rel_l2(out.cpu().numpy(), ref)
    plan.close()


def test_feather_rejects_bad_arguments():
    from paper_2609_17636_b300 import IvisError, Plan
    plan = Plan(48, 1, 1, 16, 1e-5, "fp32")  # n not a power of two
    x = torch.zeros(1, 48, 48, device="cuda")
    with pytest.raises(IvisError):
        plan.feather(x, x, 1e-3)
    plan.close()
    plan = Plan(64, 1, 1, 16, 1e-5, "fp32")
    x = torch.zeros(1, 64, 64, device="cuda")
    with pytest.raises(IvisError):
        plan.feather(x, x, -1.0)
    plan.close()
