"""Parity of the Toeplitz form of the data term (toeplitz = 1) with the FP64 oracle.

The Toeplitz form computes the same Q_tot and gradient as the visibility path (the expansion
of Eq. 6 with Eqs. 3-5 is exact), so the oracle's direct cost_grad is the reference, at the
same tolerances: relative 1e-9 (FP64) and 1e-5 (FP32). The oracle's own Toeplitz restatement
is pinned to the direct one in the CPU suite."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _data import attach_data, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5}


def _plan(prob, precision, **kw):
    from paper_2609_17636_b300 import plan_from_problem
    return plan_from_problem(prob, precision, toeplitz=True, **kw)


@pytest.fixture(scope="module")
def mosaic():
    prob = synth.small_mosaic(301, n=96, nb=64, nchan=2, npoint=3, ndump=20, n_ant=24,
                              cell_arcsec=20.0, lambda_r=0.3, lambda_s=0.5, sd_fwhm_pix=5.0)
    attach_data(prob)
    rng = np.random.default_rng(301)
    x = prob.sky_true * rng.uniform(0.3, 1.3, prob.sky_true.shape)
    f, g, terms = oracle.cost_grad(prob, x, prob.tsd, prob.sigma_sd, with_terms=True)
    return prob, x, f, g, terms


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_toeplitz_cost_and_gradient_match_oracle(mosaic, precision):
    prob, x, f, g, terms = mosaic
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.as_tensor(x, dtype=dt, device="cuda")
    fg, grad, tg = plan.cost_grad(xs)
    tol = TOL[precision]
    assert abs(fg - f) <= tol * abs(f), (fg, f)
    for a, b in zip(tg, terms):
        assert abs(a - b) <= tol * abs(b) + 1e-300, (tg, terms)
    assert rel_l2(grad.cpu().numpy(), g) <= tol, rel_l2(grad.cpu().numpy(), g)
    # the visibility path's predict still runs on a Toeplitz plan
    pair = prob.pairs[0]
    got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()
    assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair)) <= tol
    plan.close()


def test_toeplitz_needs_no_visibility_pass(mosaic):
    from paper_2609_17636_b300 import plan_from_problem
    prob, x, f, g, terms = mosaic
    pt = _plan(prob, "fp32")
    pn = plan_from_problem(prob, "fp32")
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    ft, gt, _ = pt.cost_grad(xs)
    fn, gn, _ = pn.cost_grad(xs)
    assert pt.launches_per_eval() < pn.launches_per_eval()
    assert abs(ft - fn) <= 2e-5 * abs(fn) and rel_l2(gt.cpu().numpy(), gn.cpu().numpy()) <= 2e-5
    pt.close()
    pn.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_toeplitz_edge_cases(precision):
    """Smallest window, a pair with no data, a single visibility, windows hanging off the sky,
    visibilities on grid cells and on the fold boundary, and a re-projected pointing."""
    prob = synth.small_mosaic(303, n=20, nb=16, nchan=2, npoint=3, ndump=2, n_ant=5,
                              lambda_r=0.0, lambda_s=0.0)
    prob.centres[:] = [[10, 10], [-5, 3], [18, 19]]
    for i, keep in ((1, 0), (2, 1)):
        prob.pairs[i].uvw = prob.pairs[i].uvw[:keep]
        prob.pairs[i].weight = prob.pairs[i].weight[:keep]
        prob.pairs[i].noise = prob.pairs[i].noise[:keep]
    nf = 32
    fold = 1.0 / (nf * prob.cell_rad)
    uvw = prob.pairs[3].uvw.astype(np.float64)
    uvw[:4, 0] = np.array([0.0, 3.0, -5.0, nf / 2]) * fold
    uvw[:4, 1] = np.array([0.0, -7.0, nf - 1, 2.0]) * fold
    prob.pairs[3].uvw = uvw.astype(np.float32)
    prob.grids = {2: synth.projection_grid(16, 17.6, 18.3, 0.3, 0.95, 0.05)}
    attach_data(prob)
    x = prob.sky_true * 0.5
    f, g = oracle.cost_grad(prob, x)
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fg, grad, _ = plan.cost_grad(torch.as_tensor(x, dtype=dt, device="cuda"))
    tol = TOL[precision]
    assert abs(fg - f) <= tol * abs(f)
    assert rel_l2(grad.cpu().numpy(), g) <= tol
    plan.close()


def test_toeplitz_new_data_updates_b_and_constant():
    """Setting a pair's visibilities again (same uv coverage) changes b and C: the cost and
    gradient follow the new data."""
    prob = synth.small_mosaic(305, n=48, nb=32, nchan=1, npoint=2, ndump=6, n_ant=10,
                              lambda_r=0.0, lambda_s=0.0)
    attach_data(prob)
    plan = _plan(prob, "fp64")
    x = prob.sky_true * 0.7
    xs = torch.as_tensor(x, device="cuda")
    f1, _, _ = plan.cost_grad(xs)
    assert abs(f1 - oracle.cost_grad(prob, x)[0]) <= 1e-9 * f1
    rng = np.random.default_rng(305)
    pair = prob.pairs[1]
    pair.vis = (pair.vis * 1.7 + 0.01 * rng.standard_normal(pair.m)).astype(np.complex64)
    plan.set_vis(pair.k, pair.chan, torch.as_tensor(pair.uvw, device="cuda"),
                 torch.view_as_real(torch.as_tensor(pair.vis)).cuda(),
                 torch.as_tensor(pair.weight, device="cuda"))
    f2, g2, _ = plan.cost_grad(xs)
    fr, gr = oracle.cost_grad(prob, x)
    assert abs(f2 - fr) <= 1e-9 * fr and rel_l2(g2.cpu().numpy(), gr) <= 1e-9
    plan.close()


def test_toeplitz_solve_follows_the_visibility_path():
    """The FP64 solves of the two forms see the same cost and gradient to ~1e-12, so their
    L-BFGS trajectories agree: equal final costs after 30 iterations."""
    from paper_2609_17636_b300 import plan_from_problem
    prob = synth.small_mosaic(306, n=64, nb=32, nchan=1, npoint=3, ndump=10, n_ant=16,
                              cell_arcsec=30.0, lambda_r=0.1, lambda_s=0.5, sd_fwhm_pix=4.0)
    attach_data(prob)
    pt = _plan(prob, "fp64")
    pn = plan_from_problem(prob, "fp64")
    xt = torch.zeros((1, 64, 64), dtype=torch.float64, device="cuda")
    xn = torch.zeros_like(xt)
    rt = pt.solve(xt, maxiter=30, pgtol=0.0, ftol=0.0)
    rn = pn.solve(xn, maxiter=30, pgtol=0.0, ftol=0.0)
    assert abs(rt["f"] - rn["f"]) <= 1e-6 * rn["f"], (rt, rn)
    f_or, _ = oracle.cost_grad(prob, xt.cpu().numpy(), prob.tsd, prob.sigma_sd)
    assert abs(f_or - rt["f"]) <= 1e-9 * f_or
    pt.close()
    pn.close()


def test_toeplitz_fullsize_sampled_parity():
    """The benchmark mosaic (7 pointings, 512^2 sky, nb = 512, 1.36 M visibilities, fusion and
    Laplacian on) in FP32, sparse data and evaluation skies (see test_gpu_fullsize)."""
    from paper_2609_17636_b300 import plan_from_problem
    prob = synth.config_c2()
    rng = np.random.default_rng(2024)

    def sparse(k):
        s = np.zeros((1, prob.n, prob.n))
        s.flat[rng.choice(prob.n * prob.n, size=k, replace=False)] = rng.uniform(0.2, 1.0, size=k)
        return s
    truth = sparse(48)
    for pair in prob.pairs:
        pair.vis = (oracle.pair_model_vis(prob, truth, pair) + pair.noise).astype(np.complex64)
    b = oracle.dish_kernel(prob.sd_fwhm_pix)
    t = oracle.dish_conv(truth[0], b)[None]
    prob.sigma_sd = np.array([0.05 * np.sqrt(np.mean(t ** 2))])
    prob.tsd = (t + prob.sd_noise_unit * prob.sigma_sd[0]).astype(np.float32)
    x = sparse(40)
    plan = plan_from_problem(prob, "fp32", toeplitz=True, autotune=True)
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    f, g, (Q, K, R) = plan.cost_grad(xs)
    g = g.cpu().numpy()
    resid = [oracle.pair_model_vis(prob, x, p) - p.vis.astype(np.complex128) for p in prob.pairs]
    Q_ref = sum(0.5 * float(np.sum(p.weight.astype(np.float64) * np.abs(r) ** 2))
                for p, r in zip(prob.pairs, resid))
    R_ref, gR = oracle.reg_cost_grad(x)
    K_ref, gK = oracle.fusion_cost_grad(x, prob.tsd, prob.sigma_sd, prob.sd_fwhm_pix)
    tol = TOL["fp32"]
    assert abs(Q - Q_ref) <= tol * Q_ref, (Q, Q_ref)
    assert abs(f - (Q_ref + prob.lambda_s * K_ref + prob.lambda_r * R_ref)) <= tol * f
    ys = np.concatenate([rng.integers(0, prob.n, 40), [0, prob.n - 1, 256, 256]])
    xs_ = np.concatenate([rng.integers(0, prob.n, 40), [5, prob.n - 1, 256, 410]])
    gq = oracle.data_grad_pixels(prob, x, 0, ys, xs_, residuals=resid)
    g_ref = gq + prob.lambda_r * gR[0, ys, xs_] + prob.lambda_s * gK[0, ys, xs_]
    assert rel_l2(g[0, ys, xs_], g_ref) <= tol, rel_l2(g[0, ys, xs_], g_ref)
    plan.close()


def test_toeplitz_config_limits():
    from paper_2609_17636_b300 import IvisError, Plan
    with pytest.raises(IvisError):
        Plan(4096, 1, 1, 2048, 1e-5, "fp32", toeplitz=True)
    with pytest.raises(IvisError):
        Plan(64, 1, 1, 32, 1e-5, "fp64", toeplitz=True, serial_pairs=True)
