"""Parity at full sizes: the 7-pointing 512^2 mosaic (1.36 M visibilities, Laplacian +
fusion terms, FP32 grids) and the batched cube (36 beams x 32 channels, 1152 pairs, ragged
U[1e5, 3e5] visibilities per pair, 2.3e8 in all), in the launch configuration bench.py times
(the autotuned plan's captured evaluation graph).

The oracle cannot evaluate a dense 512^2 sky against 1.36 M visibilities in seconds, so both
the data and the evaluation point are sparse skies (the oracle's direct DFT skips zero
pixels, which leaves its sums unchanged): then the oracle's cost terms are exact and cheap,
and the gradient is checked on sampled pixels and the model visibilities on sampled rows.
Tolerance: the FP32 path's 1e-5 relative."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _data import rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _sparse_sky(rng, n, k, lo=0.0):
    sky = np.zeros((1, n, n))
    idx = rng.choice(n * n, size=k, replace=False)
    sky.flat[idx] = rng.uniform(0.2, 1.0, size=k) + lo
    return sky


@pytest.fixture(scope="module")
def c2():
    prob = synth.config_c2()
    rng = np.random.default_rng(2024)
    truth = _sparse_sky(rng, prob.n, 48)
    for pair in prob.pairs:
        pair.vis = (oracle.pair_model_vis(prob, truth, pair) + pair.noise).astype(np.complex64)
    b = oracle.dish_kernel(prob.sd_fwhm_pix)
    t = oracle.dish_conv(truth[0], b)[None]
    prob.sigma_sd = np.array([0.05 * np.sqrt(np.mean(t ** 2))])
    prob.tsd = (t + prob.sd_noise_unit * prob.sigma_sd[0]).astype(np.float32)
    x = _sparse_sky(rng, prob.n, 40)
    return prob, x


def test_fullsize_cost_terms_gradient_samples_and_visibilities(c2):
    """In the bench's launch configuration: FP32 plan with the autotuner's chunk size and
    column width, evaluation through the captured graph."""
    from paper_2609_17636_b300 import plan_from_problem
    prob, x = c2
    plan = plan_from_problem(prob, "fp32", autotune=True)
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    f, g, (Q, K, R) = plan.cost_grad(xs)
    g = g.cpu().numpy()
    # oracle terms
    resid = [oracle.pair_model_vis(prob, x, p) - p.vis.astype(np.complex128) for p in prob.pairs]
    Q_ref = sum(0.5 * float(np.sum(p.weight.astype(np.float64) * np.abs(r) ** 2))
                for p, r in zip(prob.pairs, resid))
    R_ref, gR = oracle.reg_cost_grad(x)
    K_ref, gK = oracle.fusion_cost_grad(x, prob.tsd, prob.sigma_sd, prob.sd_fwhm_pix)
    f_ref = Q_ref + prob.lambda_s * K_ref + prob.lambda_r * R_ref
    assert abs(Q - Q_ref) <= TOL * Q_ref
    assert abs(K - K_ref) <= TOL * K_ref
    assert abs(R - R_ref) <= TOL * R_ref
    assert abs(f - f_ref) <= TOL * f_ref
    # gradient at sampled pixels: inside several windows, on the sky edge, in overlaps
    rng = np.random.default_rng(7)
    ys = np.concatenate([rng.integers(0, prob.n, 40), [0, prob.n - 1, 256, 256]])
    xs_ = np.concatenate([rng.integers(0, prob.n, 40), [5, prob.n - 1, 256, 410]])
    gq = oracle.data_grad_pixels(prob, x, 0, ys, xs_, residuals=resid)
    g_ref = gq + prob.lambda_r * gR[0, ys, xs_] + prob.lambda_s * gK[0, ys, xs_]
    assert rel_l2(g[0, ys, xs_], g_ref) <= TOL, rel_l2(g[0, ys, xs_], g_ref)
    # model visibilities on sampled rows of every pointing
    for pair in prob.pairs:
        idx = np.sort(rng.choice(pair.m, 1500, replace=False))
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()[idx]
        ref = oracle.pair_model_vis(prob, x, pair, idx)
        assert rel_l2(got[:, 0] + 1j * got[:, 1], ref) <= TOL
    plan.close()


def test_fullsize_gradient_is_consistent_with_cost_along_a_direction(c2):
    """Directional derivative by central differences of the GPU cost (a property that holds at
    any size) on a dense random sky: (f(x + h d) - f(x - h d)) / 2h = <g, d>."""
    from paper_2609_17636_b300 import plan_from_problem
    prob, _ = c2
    plan = plan_from_problem(prob, "fp64")
    rng = np.random.default_rng(3)
    x = torch.as_tensor(prob.sky_true * rng.uniform(0.5, 1.5, prob.sky_true.shape), device="cuda")
    d = torch.as_tensor(rng.standard_normal(prob.sky_true.shape), device="cuda")
    _, g, _ = plan.cost_grad(x)
    h = 0.05 * float(x.abs().max()) / float(d.abs().max())  # the cost is quadratic: no truncation error
    fp, _, _ = plan.cost_grad(x + h * d)
    fm, _, _ = plan.cost_grad(x - h * d)
    fd = (fp - fm) / (2 * h)
    ip = float(torch.sum(g * d))
    assert abs(fd - ip) <= 1e-6 * abs(ip)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_maximum_window_size_sampled_parity(precision):
    """nb = 2048 (the largest window; 4096^2 fine grid, radix-16 FFT passes of length 4096,
    16384 tiles per pair): two pointings of the full-footprint geometry on a 4096^2 sky at
    5 arcsec with 630 x 400 visibilities each; sparse data and evaluation skies as above."""
    from paper_2609_17636_b300 import plan_from_problem
    prob = synth.config_c4(dumps=400)
    prob.centres = prob.centres[[14, 21]]
    prob.beams = prob.beams[:2]
    prob.pairs = [p for p in prob.pairs if p.k in (14, 21)]
    for i, p in enumerate(prob.pairs):
        p.k = i
    prob.lambda_s = 0.0
    rng = np.random.default_rng(11)
    truth = _sparse_sky(rng, prob.n, 30)
    for pair in prob.pairs:
        pair.vis = (oracle.pair_model_vis(prob, truth, pair) + pair.noise).astype(np.complex64)
    x = _sparse_sky(rng, prob.n, 25)
    plan = plan_from_problem(prob, precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    xs = torch.as_tensor(x, dtype=dt, device="cuda")
    f, g, (Q, K, R) = plan.cost_grad(xs)
    tol = 1e-5 if precision == "fp32" else 1e-9
    resid = [oracle.pair_model_vis(prob, x, p) - p.vis.astype(np.complex128) for p in prob.pairs]
    Q_ref = sum(0.5 * float(np.sum(p.weight.astype(np.float64) * np.abs(r) ** 2))
                for p, r in zip(prob.pairs, resid))
    R_ref, gR = oracle.reg_cost_grad(x)
    assert abs(Q - Q_ref) <= tol * Q_ref and abs(R - R_ref) <= tol * R_ref
    ys = rng.integers(0, prob.n, 24)
    xs_ = rng.integers(0, prob.n, 24)
    ys[:4], xs_[:4] = prob.centres[0][1] + np.array([0, 5, -700, 1000]), prob.centres[0][0] + np.array([0, 3, 900, -1020])
    gq = oracle.data_grad_pixels(prob, x, 0, ys, xs_, residuals=resid)
    g_ref = gq + prob.lambda_r * gR[0, ys, xs_]
    assert rel_l2(g.cpu().numpy()[0, ys, xs_], g_ref) <= tol
    for pair in prob.pairs:
        idx = np.sort(rng.choice(pair.m, 800, replace=False))
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()[idx]
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair, idx)) <= tol
    plan.close()


def test_batched_cube_sampled_parity():
    """The batched cube at its full size and in the bench's launch configuration: 36 beams on
    the 6 x 6 hexagonal footprint (0.9 deg pitch, 1 deg beams, 512^2 windows on a 1024^2 sky
    at 25 arcsec, so windows overlap and hang off the sky), 32 channels (1152 pairs, uv scaled
    per channel), ragged U[1e5, 3e5] visibilities per pair that fold several times over the
    fine grid, the Laplacian term; the FP32 plan with the autotuner's tile and item choice.
    Sparse data and evaluation skies per channel as above."""
    from paper_2609_17636_b300 import plan_from_problem
    prob = synth.config_c3()
    assert len(prob.pairs) == 1152 and min(p.m for p in prob.pairs) >= 100_000
    rng = np.random.default_rng(3003)
    truth = np.concatenate([_sparse_sky(rng, prob.n, 24) for _ in range(prob.nchan)])
    for pair in prob.pairs:
        pair.vis = (oracle.pair_model_vis(prob, truth, pair) + pair.noise).astype(np.complex64)
    x = np.concatenate([_sparse_sky(rng, prob.n, 20) for _ in range(prob.nchan)])
    plan = plan_from_problem(prob, "fp32", autotune=True)
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    f, g, (Q, K, R) = plan.cost_grad(xs)
    g = g.cpu().numpy()
    resid = [oracle.pair_model_vis(prob, x, p) - p.vis.astype(np.complex128) for p in prob.pairs]
    Q_ref = sum(0.5 * float(np.sum(p.weight.astype(np.float64) * np.abs(r) ** 2))
                for p, r in zip(prob.pairs, resid))
    R_ref, gR = oracle.reg_cost_grad(x)
    f_ref = Q_ref + prob.lambda_r * R_ref
    assert abs(Q - Q_ref) <= TOL * Q_ref and abs(R - R_ref) <= TOL * R_ref and K == 0.0
    assert abs(f - f_ref) <= TOL * f_ref
    # gradient at sampled pixels of two channels: random, beam centres (overlaps), sky corners
    for chan in (0, 17, 31):
        ys = np.concatenate([rng.integers(0, prob.n, 30), prob.centres[::5, 1], [0, prob.n - 1]])
        xx = np.concatenate([rng.integers(0, prob.n, 30), prob.centres[::5, 0], [prob.n - 1, 0]])
        sub = [(i, p) for i, p in enumerate(prob.pairs) if p.chan == chan]
        gq = oracle.data_grad_pixels(prob, x, chan, ys, xx,
                                     residuals={i: resid[i] for i, _ in sub})
        g_ref = gq + prob.lambda_r * gR[chan, ys, xx]
        assert rel_l2(g[chan, ys, xx], g_ref) <= TOL, (chan, rel_l2(g[chan, ys, xx], g_ref))
    for pair in prob.pairs[::97]:
        idx = np.sort(rng.choice(pair.m, 1000, replace=False))
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()[idx]
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair, idx)) <= TOL
    plan.close()
