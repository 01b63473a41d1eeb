"""Parity of the w-stacked full visibility equation (wterm = 1, Eq. 1 with the w-term and
1/n) with the oracle's direct evaluation of Eq. 1, at the path tolerances: relative 1e-9 (FP64)
and 1e-5 (FP32) on the cost, its terms, the gradient and model visibilities."""
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
    return plan_from_problem(prob, precision, **kw)


@pytest.fixture(scope="module")
def wide():
    """A wide-field mosaic: 64^2 windows of 1 arcmin cells (windows reach 0.76 deg from their
    centres), 16 antennas over 6 km, 12 dumps over +-4 h: |w (n - 1)| reaches ~2 turns."""
    prob = synth.small_mosaic(401, n=96, nb=64, nchan=2, npoint=3, ndump=12, n_ant=16,
                              cell_arcsec=60.0, lambda_r=0.3, lambda_s=0.5, sd_fwhm_pix=5.0)
    prob.wterm = True
    attach_data(prob)
    rng = np.random.default_rng(401)
    x = prob.sky_true * rng.uniform(0.3, 1.3, prob.sky_true.shape)
    f, g, terms = oracle.cost_grad(prob, x, prob.tsd, prob.sigma_sd, with_terms=True)
    return prob, x, f, g, terms


def test_the_wterm_matters_in_this_geometry(wide):
    prob, x, *_ = wide
    pair = prob.pairs[0]
    vw = oracle.pair_model_vis(prob, x, pair)
    prob.wterm = False
    vc = oracle.pair_model_vis(prob, x, pair)
    prob.wterm = True
    assert rel_l2(vc, vw) > 0.1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_wterm_cost_gradient_and_visibilities_match_oracle(wide, precision):
    prob, x, f, g, terms = wide
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.as_tensor(x, dtype=dt, device="cuda")
    fg, grad, tg = plan.cost_grad(xs)
    tol = TOL[precision]
    assert abs(fg - f) <= tol * abs(f), (fg, f)
    for a, b in zip(tg, terms):
        assert abs(a - b) <= tol * abs(b) + 1e-300, (tg, terms)
    assert rel_l2(grad.cpu().numpy(), g) <= tol, rel_l2(grad.cpu().numpy(), g)
    for pair in prob.pairs[:4]:
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair)) <= tol
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_wterm_edge_cases(precision):
    """Constant w in one pair (the fewest planes), an empty pair, a single visibility, windows
    off the sky edge, a re-projected pointing."""
    prob = synth.small_mosaic(403, n=40, nb=32, nchan=1, npoint=3, ndump=4, n_ant=8,
                              cell_arcsec=90.0, lambda_r=0.0, lambda_s=0.0)
    prob.wterm = True
    prob.centres[:] = [[20, 20], [-6, 5], [37, 36]]
    uvw = prob.pairs[0].uvw.copy()
    uvw[:, 2] = 1234.5
    prob.pairs[0].uvw = uvw
    prob.pairs[1].uvw = prob.pairs[1].uvw[:0]
    prob.pairs[1].weight = prob.pairs[1].weight[:0]
    prob.pairs[1].noise = prob.pairs[1].noise[:0]
    prob.pairs[2].uvw = prob.pairs[2].uvw[:1]
    prob.pairs[2].weight = prob.pairs[2].weight[:1]
    prob.pairs[2].noise = prob.pairs[2].noise[:1]
    prob.grids = {2: synth.projection_grid(32, 36.4, 35.7, 0.25, 1.02, 0.03)}
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


def test_wterm_solve_and_restrictions(wide):
    from paper_2609_17636_b300 import IvisError, Plan, dirty_image
    prob, *_ = wide
    plan = _plan(prob, "fp64")
    x = torch.zeros(prob.sky_true.shape, dtype=torch.float64, device="cuda")
    rep = plan.solve(x, maxiter=15, pgtol=0.0, ftol=0.0)
    f_or, _ = oracle.cost_grad(prob, x.cpu().numpy(), prob.tsd, prob.sigma_sd)
    assert abs(f_or - rep["f"]) <= 1e-9 * f_or
    with pytest.raises(IvisError):
        dirty_image(plan)
    plan.close()
    with pytest.raises(IvisError):
        Plan(64, 1, 1, 32, 1e-4, "fp32", wterm=True, toeplitz=True)


def test_wterm_fullsize_sampled_parity():
    """The benchmark mosaic (7 pointings, 512^2 sky at 7 arcsec, nb = 512, 1.36 M
    visibilities) with the full Eq. 1, FP32, sparse data and evaluation skies (the oracle's
    direct sums skip zero pixels): cost terms, sampled gradient pixels, sampled visibilities."""
    prob = synth.config_c2()
    prob.wterm = True
    prob.lambda_s = 0.0
    rng = np.random.default_rng(77)

    def sparse(k):
        s = np.zeros((1, prob.n, prob.n))
        s.flat[rng.choice(prob.n * prob.n, size=k, replace=False)] = rng.uniform(0.2, 1.0, size=k)
        return s
    truth = sparse(40)
    for pair in prob.pairs:
        pair.vis = (oracle.pair_model_vis(prob, truth, pair) + pair.noise).astype(np.complex64)
    x = sparse(30)
    plan = _plan(prob, "fp32")
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    f, g, (Q, K, R) = plan.cost_grad(xs)
    resid = [oracle.pair_model_vis(prob, x, p) - p.vis.astype(np.complex128) for p in prob.pairs]
    Q_ref = sum(0.5 * float(np.sum(p.weight.astype(np.float64) * np.abs(r) ** 2))
                for p, r in zip(prob.pairs, resid))
    R_ref, gR = oracle.reg_cost_grad(x)
    assert abs(Q - Q_ref) <= 1e-5 * Q_ref and abs(R - R_ref) <= 1e-5 * R_ref
    ys = np.concatenate([rng.integers(0, prob.n, 30), [0, 256, 511]])
    xs_ = np.concatenate([rng.integers(0, prob.n, 30), [0, 256, 300]])
    gq = oracle.data_grad_pixels(prob, x, 0, ys, xs_, residuals=resid)
    g_ref = gq + prob.lambda_r * gR[0, ys, xs_]
    assert rel_l2(g.cpu().numpy()[0, ys, xs_], g_ref) <= 1e-5
    for pair in prob.pairs[:3]:
        idx = np.sort(rng.choice(pair.m, 1000, replace=False))
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()[idx]
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair, idx)) <= 1e-5
    plan.close()
