"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated by the method's targets): relative L2 <= 1e-9 for the FP64 path and
<= 1e-5 for the FP32 path, on model visibilities and on the gradient; the cost and its three
terms to the same relative bound. Inputs are seeded synthetic problems whose data come from
the oracle (tests/_data.py)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _data import attach_data, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5}


@pytest.fixture(scope="module")
def mosaic():
    """3 pointings x 2 channels, 96^2 sky, 64^2 windows off the sky edges, 24 antennas x
    20 dumps (ragged per pair after flagging), baselines far beyond the pixel Nyquist limit
    (the NUFFT folds), Laplacian and fusion terms on."""
    prob = synth.small_mosaic(301, n=96, nb=64, nchan=2, npoint=3, ndump=20, n_ant=24,
                              cell_arcsec=20.0, lambda_r=0.3, lambda_s=0.5, sd_fwhm_pix=5.0)
    attach_data(prob)
    rng = np.random.default_rng(301)
    x = prob.sky_true * rng.uniform(0.3, 1.3, prob.sky_true.shape)
    f, g, terms = oracle.cost_grad(prob, x, prob.tsd, prob.sigma_sd, with_terms=True)
    return prob, x, f, g, terms


def _plan(prob, precision, **kw):
    from paper_2609_17636_b300 import plan_from_problem
    return plan_from_problem(prob, precision, **kw)


@pytest.mark.parametrize("precision,tile,kern", [("fp64", 0, 0), ("fp32", 32, 1), ("fp32", 64, 1),
                                                 ("fp32", 32, 2), ("fp32", 64, 2)])
def test_cost_and_gradient_match_oracle(mosaic, precision, tile, kern):
    """FP32 runs the scalar item pass (kern 1: one lane per kernel column) and the tensor-core
    item pass (kern 2: split-TF32 mma per 8 x 8 block) with 32- and 64-cell tiles (the 128^2
    fine grids hold 2 x 2 tiles of 64 cells, each patch wrapping at the grid edge)."""
    prob, x, f, g, terms = mosaic
    plan = _plan(prob, precision, grid_tile=tile, grid_kernel=kern)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.as_tensor(x, dtype=dt, device="cuda")
    fg, grad, tg = plan.cost_grad(xs)
    tol = TOL[precision]
    assert abs(fg - f) <= tol * abs(f), (fg, f)
    for a, b in zip(tg, terms):
        assert abs(a - b) <= tol * abs(b) + 1e-300, (tg, terms)
    assert rel_l2(grad.cpu().numpy(), g) <= tol, rel_l2(grad.cpu().numpy(), g)
    plan.close()


@pytest.mark.parametrize("width", [3, 5, 8])
def test_item_passes_at_other_kernel_widths(mosaic, width):
    """The scalar and tensor-core item passes at kernel widths 3, 5 and 8 (a quad's lanes then
    hold one or two taps each, and the footprint of an 8 x 8 block fills 10 to 15 of its 16 rows
    and columns): both within the NUFFT's error of the oracle (about 10^-(W - 1)), and the same
    cost and gradient to FP32 rounding."""
    prob, x, f, g, terms = mosaic
    res = {}
    for kern in (1, 2):
        plan = _plan(prob, "fp32", kernel_width=width, grid_kernel=kern)
        fg, grad, _ = plan.cost_grad(torch.as_tensor(x, dtype=torch.float32, device="cuda"))
        res[kern] = (fg, grad.cpu().numpy())
        plan.close()
    bound = max(TOL["fp32"], 10.0 ** -(width - 2))
    for fg, gr in res.values():
        assert abs(fg - f) <= bound * abs(f), (fg, f)
        assert rel_l2(gr, g) <= bound
    assert abs(res[1][0] - res[2][0]) <= 2e-6 * abs(res[1][0]), (res[1][0], res[2][0])
    assert rel_l2(res[2][1], res[1][1]) <= 2e-6, rel_l2(res[2][1], res[1][1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_repeated_evaluations_leave_no_state(precision):
    """Evaluations at x1, x2, x1 on a plan with an odd number of (pointing, channel) slots, so
    that the last two-window transform has an empty partner: the third result equals the first
    and both match the oracle. Each evaluation writes the forward grids' Hermitian halves,
    folds the adjoint grids onto theirs, reads them and clears them for the next one; a grid
    left uncleared would add the previous evaluation's data term."""
    prob = synth.small_mosaic(77, n=96, nb=64, nchan=1, npoint=3, ndump=16, n_ant=20,
                              cell_arcsec=20.0, lambda_r=0.1, lambda_s=0.0)
    attach_data(prob)
    assert len([p for p in prob.pairs if p.m > 0]) % 2 == 1
    rng = np.random.default_rng(78)
    x1 = prob.sky_true * rng.uniform(0.5, 1.5, prob.sky_true.shape)
    x2 = prob.sky_true * rng.uniform(0.0, 2.0, prob.sky_true.shape)
    f_ref, g_ref = oracle.cost_grad(prob, x1, prob.tsd, prob.sigma_sd)
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    f1, g1, _ = plan.cost_grad(torch.as_tensor(x1, dtype=dt, device="cuda"))
    g1 = g1.cpu().numpy()
    plan.cost_grad(torch.as_tensor(x2, dtype=dt, device="cuda"))
    f3, g3, _ = plan.cost_grad(torch.as_tensor(x1, dtype=dt, device="cuda"))
    g3 = g3.cpu().numpy()
    tol = TOL[precision]
    assert abs(f1 - f_ref) <= tol * abs(f_ref) and rel_l2(g1, g_ref) <= tol
    # the cost partials are summed in a fixed order; the gradient's spreading reductions are
    # atomic, so only their order can differ between evaluations
    assert f3 == f1
    assert rel_l2(g3, g1) <= (1e-13 if precision == "fp64" else 1e-6), rel_l2(g3, g1)
    plan.close()


def test_serial_pairs_path_matches_oracle_and_batched_path(mosaic):
    """The unbatched FP64 path (one pair per launch sequence) used as the solver baseline."""
    from paper_2609_17636_b300 import plan_from_problem
    prob, x, f, g, terms = mosaic
    xs = torch.as_tensor(x, device="cuda")
    ps = plan_from_problem(prob, "fp64", serial_pairs=True)
    pb = plan_from_problem(prob, "fp64")
    fs, gs, _ = ps.cost_grad(xs)
    fb, gb, _ = pb.cost_grad(xs)
    assert abs(fs - f) <= 1e-9 * abs(f) and rel_l2(gs.cpu().numpy(), g) <= 1e-9
    assert abs(fs - fb) <= 1e-12 * abs(fb) and rel_l2(gs.cpu().numpy(), gb.cpu().numpy()) <= 1e-12
    assert ps.launches_per_eval() > pb.launches_per_eval()
    ps.close()
    pb.close()


def test_autotuned_plan_matches_oracle_and_caches_its_choice(mosaic, tmp_path, monkeypatch):
    from paper_2609_17636_b300 import plan_from_problem
    prob, x, f, g, terms = mosaic
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("IVIS_AUTOTUNE_CACHE", str(cache))
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    p1 = plan_from_problem(prob, "fp32", autotune=True)
    f1, g1, _ = p1.cost_grad(xs)
    t1 = p1.tuning()
    assert t1["chunk_cap"] in (256, 512, 1024, 2048, 4096) and t1["fft_cols"] in (1, 2, 4, 8, 16)
    assert ("tile 32," in t1["decision"]) != ("tile 64," in t1["decision"])
    if "tile 32," in t1["decision"]:
        assert t1["chunk_cap"] <= 2048
    else:
        assert t1["chunk_cap"] >= 1024
    assert "(timed)" in t1["decision"] and cache.read_text().count("|") == 1
    assert abs(f1 - f) <= TOL["fp32"] * abs(f) and rel_l2(g1.cpu().numpy(), g) <= TOL["fp32"]
    p2 = plan_from_problem(prob, "fp32", autotune=True)
    p2.prepare()
    t2 = p2.tuning()
    assert "(cached)" in t2["decision"] and t2["chunk_cap"] == t1["chunk_cap"]
    assert t2["decision"].split("->")[1].split(", fft")[0] == t1["decision"].split("->")[1].split(", fft")[0]
    p1.close()
    p2.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_model_visibilities_match_direct_dft(mosaic, precision):
    prob, x, *_ = mosaic
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.as_tensor(x, dtype=dt, device="cuda")
    for pair in prob.pairs:
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()
        got = got[:, 0] + 1j * got[:, 1]
        ref = oracle.pair_model_vis(prob, x, pair)
        assert rel_l2(got, ref) <= TOL[precision], (pair.k, pair.chan, rel_l2(got, ref))
    plan.close()


def test_single_dish_model_matches_oracle(mosaic):
    prob, x, *_ = mosaic
    plan = _plan(prob, "fp64")
    got = plan.sd_predict(torch.as_tensor(x, device="cuda")).cpu().numpy()
    b = oracle.dish_kernel(prob.sd_fwhm_pix)
    ref = np.stack([oracle.dish_conv(x[c], b) for c in range(prob.nchan)])
    assert rel_l2(got, ref) <= 1e-12
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_dish_wide_beam_matches_oracle(precision):
    """The 16 arcmin dish at 7 arcsec (FWHM 137 px, 467 taps) on a 256^2 sky: the taps run
    past the image on both sides; the fused residual/K path against the oracle's K."""
    from paper_2609_17636_b300 import Plan
    rng = np.random.default_rng(5)
    n, fwhm = 256, 16 * 60 / 7.0
    sky = rng.uniform(0, 1, (1, n, n))
    b = oracle.dish_kernel(fwhm)
    tsd = oracle.dish_conv(sky[0] * 0.8, b)[None] + 0.01 * rng.standard_normal((1, n, n))
    tsd = tsd.astype(np.float32)
    plan = Plan(n, 1, 1, 16, 1e-5, precision, lambda_s=0.7)
    plan.set_pointing(0, n // 2, n // 2, torch.ones(16, 16, device="cuda"))
    plan.set_vis(0, 0, torch.zeros((0, 3), device="cuda"), None, None)
    plan.set_sd(0, torch.as_tensor(tsd[0], device="cuda"), 0.05, fwhm)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.as_tensor(sky, dtype=dt, device="cuda")
    f, g, terms = plan.cost_grad(xs)
    K, gK = oracle.fusion_cost_grad(sky, tsd, 0.05, fwhm)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert abs(terms[1] - K) <= tol * K and abs(f - 0.7 * K) <= tol * f
    assert rel_l2(g.cpu().numpy(), 0.7 * gK) <= tol
    assert rel_l2(plan.sd_predict(xs).cpu().numpy()[0], oracle.dish_conv(sky[0], b)) <= tol
    plan.close()


def test_gradient_central_differences_fp64(mosaic):
    prob, x, *_ = mosaic
    plan = _plan(prob, "fp64")
    xs = torch.as_tensor(x, device="cuda")
    _, g, _ = plan.cost_grad(xs)
    g = g.cpu().numpy()
    rng = np.random.default_rng(7)
    h = 1e-4 * np.abs(x).max()
    for i in rng.choice(x.size, 12, replace=False):
        e = torch.zeros_like(xs).view(-1)
        e[i] = h
        fp, _, _ = plan.cost_grad(xs + e.view_as(xs))
        fm, _, _ = plan.cost_grad(xs - e.view_as(xs))
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g.flat[i]) <= 1e-6 * np.abs(g).max(), (i, fd, g.flat[i])
    plan.close()


def test_data_term_quadratic_identity_fp32():
    """With V = 0 and lambda = 0, Q(x) = 1/2 ||A x||_W^2 and grad Q = A^H W A x, so
    <x, grad Q(x)> = 2 Q(x) exactly for an operator and its exact adjoint."""
    prob = synth.small_mosaic(302, n=80, nb=64, nchan=1, npoint=2, ndump=10, n_ant=20,
                              lambda_r=0.0, lambda_s=0.0)
    for p in prob.pairs:
        p.vis = np.zeros(p.m, np.complex64)
    plan = _plan(prob, "fp32")
    xs = torch.as_tensor(prob.sky_true, dtype=torch.float32, device="cuda")
    f, g, _ = plan.cost_grad(xs)
    ip = float(torch.sum(xs.double() * g.double()))
    assert abs(ip - 2 * f) <= 1e-5 * abs(2 * f)
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_cases(precision):
    """nb = 16 (smallest window), a pair with no data, a single visibility, a window that
    hangs mostly off the sky, visibilities exactly on grid cells and on the fold boundary."""
    prob = synth.small_mosaic(303, n=20, nb=16, nchan=2, npoint=3, ndump=2, n_ant=5,
                              lambda_r=0.0, lambda_s=0.0)
    prob.centres[:] = [[10, 10], [-5, 3], [18, 19]]
    prob.pairs[1].uvw = prob.pairs[1].uvw[:0]
    prob.pairs[1].weight = prob.pairs[1].weight[:0]
    prob.pairs[1].noise = prob.pairs[1].noise[:0]
    prob.pairs[2].uvw = prob.pairs[2].uvw[:1]
    prob.pairs[2].weight = prob.pairs[2].weight[:1]
    prob.pairs[2].noise = prob.pairs[2].noise[:1]
    nf = 32
    fold = 1.0 / (nf * prob.cell_rad)  # one fine-grid cell in wavelengths
    uvw = prob.pairs[3].uvw.astype(np.float64)
    uvw[:4, 0] = np.array([0.0, 3.0, -5.0, nf / 2]) * fold
    uvw[:4, 1] = np.array([0.0, -7.0, nf - 1, 2.0]) * fold
    prob.pairs[3].uvw = uvw.astype(np.float32)
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dense_single_tile_many_chunks(precision):
    """nb = 16 gives a 32^2 fine grid, i.e. a single 32-cell tile: ~3000 visibilities per pair
    split into several chunks, with many visibilities sharing a first-tap cell (the spread's
    run merging) and a ragged last chunk."""
    prob = synth.small_mosaic(304, n=24, nb=16, nchan=1, npoint=2, ndump=4, n_ant=40,
                              cell_arcsec=30.0, lambda_r=0.0, lambda_s=0.0)
    attach_data(prob)
    assert max(p.m for p in prob.pairs) > 2048
    x = prob.sky_true * 0.6
    f, g = oracle.cost_grad(prob, x)
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fg, grad, _ = plan.cost_grad(torch.as_tensor(x, dtype=dt, device="cuda"))
    tol = TOL[precision]
    assert abs(fg - f) <= tol * abs(f)
    assert rel_l2(grad.cpu().numpy(), g) <= tol
    for pair in prob.pairs:
        got = plan.predict(torch.as_tensor(x, dtype=dt, device="cuda"), pair.k, pair.chan).cpu().numpy()
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair)) <= tol
    plan.close()


@pytest.mark.parametrize("tile,kern", [(32, 1), (64, 1), (32, 2), (64, 2)])
def test_dense_single_64_cell_tile_many_chunks(tile, kern):
    """nb = 32 gives a 64^2 fine grid: one 64-cell tile (or four 32-cell tiles) holding ~6000
    visibilities per pair, split into several chunks with a ragged last one; first taps on
    every cell row and column including the wrap at the grid edge."""
    prob = synth.small_mosaic(306, n=40, nb=32, nchan=1, npoint=2, ndump=8, n_ant=40,
                              cell_arcsec=30.0, lambda_r=0.0, lambda_s=0.0)
    attach_data(prob)
    assert max(p.m for p in prob.pairs) > 4096
    x = prob.sky_true * 0.6
    f, g = oracle.cost_grad(prob, x)
    plan = _plan(prob, "fp32", grid_tile=tile, grid_kernel=kern)
    xs = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    fg, grad, _ = plan.cost_grad(xs)
    assert abs(fg - f) <= TOL["fp32"] * abs(f)
    assert rel_l2(grad.cpu().numpy(), g) <= TOL["fp32"]
    for pair in prob.pairs:
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair)) <= TOL["fp32"]
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dirty_image_and_beam_weight_map(mosaic, precision):
    """Inputs of the learned warm start: -grad Q(0) (the data term alone) and sum_k A_k^2."""
    from paper_2609_17636_b300 import dirty_image
    prob, *_ = mosaic
    plan = _plan(prob, precision)
    d, b = dirty_image(plan)
    _, gq = oracle.data_cost_grad(prob, np.zeros_like(prob.sky_true))
    assert rel_l2(d.cpu().numpy(), -gq) <= TOL[precision]
    bw = sum(oracle.window_adjoint(np.asarray(prob.beams[k], np.float64) ** 2, *prob.centres[k], (prob.n, prob.n))
             for k in range(prob.npoint))
    assert rel_l2(b.cpu().numpy(), bw) <= TOL[precision]
    plan.close()


@pytest.fixture(scope="module")
def gridded():
    """The paper's general re-projection (Eq. 2): two of three pointings sample the sky through
    rotated, scaled, slightly curved grids with fractional centres (one extends off the sky,
    one entry is NaN); the third keeps its integer window."""
    prob = synth.small_mosaic(305, n=96, nb=64, nchan=2, npoint=3, ndump=12, n_ant=20,
                              cell_arcsec=20.0, lambda_r=0.3, lambda_s=0.0)
    g0 = synth.projection_grid(64, 40.3, 47.8, rot_rad=0.25, scale=1.05, curvature=0.04)
    g1 = synth.projection_grid(64, 80.6, 20.1, rot_rad=-0.4, scale=0.93)
    g1[5, 7] = np.nan
    prob.grids = {0: g0, 1: g1}
    attach_data(prob)
    rng = np.random.default_rng(305)
    x = prob.sky_true * rng.uniform(0.3, 1.3, prob.sky_true.shape)
    f, g = oracle.cost_grad(prob, x)
    return prob, x, f, g


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_reprojection_grids_match_oracle(gridded, precision):
    from paper_2609_17636_b300 import dirty_image
    prob, x, f, g = gridded
    plan = _plan(prob, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.as_tensor(x, dtype=dt, device="cuda")
    fg, grad, _ = plan.cost_grad(xs)
    tol = TOL[precision]
    assert abs(fg - f) <= tol * abs(f)
    assert rel_l2(grad.cpu().numpy(), g) <= tol
    for pair in prob.pairs[:3]:
        got = plan.predict(xs, pair.k, pair.chan).cpu().numpy()
        assert rel_l2(got[:, 0] + 1j * got[:, 1], oracle.pair_model_vis(prob, x, pair)) <= tol
    d, b = dirty_image(plan)
    _, gq = oracle.data_cost_grad(prob, np.zeros_like(x))
    assert rel_l2(d.cpu().numpy(), -gq) <= tol
    bw = sum(oracle.pointing_window_adjoint(prob, np.asarray(prob.beams[k], np.float64) ** 2, k, (prob.n, prob.n))
             for k in range(prob.npoint))
    assert rel_l2(b.cpu().numpy(), bw) <= tol
    plan.close()


def test_invalid_inputs_are_rejected():
    from paper_2609_17636_b300 import IvisError, Plan
    plan = Plan(32, 1, 1, 16, 1e-4, "fp32")
    plan.set_pointing(0, 16, 16, torch.ones(16, 16, device="cuda"))
    uvw = torch.zeros(4, 3, device="cuda")
    vis = torch.zeros(4, 2, device="cuda")
    w = torch.ones(4, device="cuda")
    w[2] = float("nan")
    with pytest.raises(IvisError) as e:
        plan.set_vis(0, 0, uvw, vis, w)
    assert e.value.status == 6
    with pytest.raises(IvisError) as e:  # the pair was not set: cost refuses
        plan.cost_grad(torch.zeros(1, 32, 32, device="cuda"))
    assert e.value.status == 2
    with pytest.raises(IvisError) as e:
        plan.set_vis(3, 0, uvw, vis, torch.ones(4, device="cuda"))
    assert e.value.status == 1
    plan.close()
