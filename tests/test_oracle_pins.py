"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test targets a mistake the oracle could plausibly contain (sign of the
exponent, l/m transposed, pixel origin, a dropped weight, wrong boundary, wrong
kernel) and fails on it. None of them retypes the oracle's own formula.
"""
import math
import os

import numpy as np
import pytest
import scipy.ndimage
import scipy.optimize
import scipy.signal

import oracle
from _data import attach_data
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    rows = []
    meta = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line.startswith("#"):
            parts = line[1:].split()
            if len(parts) == 2:
                try:
                    meta[parts[0]] = float(parts[1])
                except ValueError:
                    pass
            continue
        if line:
            rows.append([float(t) for t in line.split()])
    return np.array(rows), meta


# ------------------------------------------------------------------------- forward DFT (Eq. 3)
def test_forward_on_grid_points_equals_fft2():
    """For u = a/(nb cell), v = b/(nb cell) the DFT of Eq. 3 is a 2-D FFT sample:
    V = exp(i pi (a + b)) * fft2(f)[b mod nb, a mod nb] (pixel origin at nb/2, l along x)."""
    rng = np.random.default_rng(1)
    nb, cell = 16, 1e-4
    f = rng.standard_normal((nb, nb))
    a = rng.integers(-40, 40, 60)
    b = rng.integers(-40, 40, 60)
    v = oracle.model_vis(f, cell, a / (nb * cell), b / (nb * cell))
    F = np.fft.fft2(f)
    expect = np.exp(1j * np.pi * (a + b)) * F[b % nb, a % nb]
    assert np.max(np.abs(v - expect)) <= 1e-10 * np.max(np.abs(F))


def test_forward_phase_centre_source_is_flat():
    nb, cell = 32, 3e-5
    f = np.zeros((nb, nb))
    f[nb // 2, nb // 2] = 2.5
    rng = np.random.default_rng(2)
    u, v = rng.uniform(-3e4, 3e4, 40), rng.uniform(-3e4, 3e4, 40)
    assert np.allclose(oracle.model_vis(f, cell, u, v), 2.5, rtol=0, atol=1e-13)


def test_forward_offset_source_phase_direction():
    """A source one pixel east (+l) of centre has phase -2 pi u cell: fixes sign and axis."""
    nb, cell = 8, 1e-3
    f = np.zeros((nb, nb))
    f[nb // 2, nb // 2 + 1] = 1.0
    u = np.array([250.0, 0.0, 100.0])
    v = np.array([0.0, 250.0, 0.0])
    got = oracle.model_vis(f, cell, u, v)
    # u cell = 0.25 cycle -> exp(-i pi/2) = -i ; v does not see an east offset
    assert np.allclose(got, [-1j, 1.0, np.exp(-2j * np.pi * 0.1)], atol=1e-14)


def test_forward_hermitian_and_periodic():
    rng = np.random.default_rng(3)
    nb, cell = 24, 2e-5
    f = rng.standard_normal((nb, nb))
    u, v = rng.uniform(-2e4, 2e4, 30), rng.uniform(-2e4, 2e4, 30)
    a = oracle.model_vis(f, cell, u, v)
    b = oracle.model_vis(f, cell, -u, -v)
    assert np.allclose(b, np.conj(a), rtol=0, atol=1e-10 * np.abs(a).max())
    c = oracle.model_vis(f, cell, u + 1.0 / cell, v - 2.0 / cell)
    assert np.allclose(c, a, rtol=0, atol=1e-9 * np.abs(a).max())


def test_forward_linear_and_sparse_skip_consistent():
    rng = np.random.default_rng(4)
    nb, cell = 16, 5e-5
    f1 = rng.standard_normal((nb, nb))
    f2 = np.zeros((nb, nb))
    f2[3, 5] = 1.7
    u, v = rng.uniform(-1e4, 1e4, 25), rng.uniform(-1e4, 1e4, 25)
    lhs = oracle.model_vis(f1 + 3 * f2, cell, u, v)
    rhs = oracle.model_vis(f1, cell, u, v) + 3 * oracle.model_vis(f2, cell, u, v)
    assert np.allclose(lhs, rhs, atol=1e-11)


def test_forward_and_adjoint_brute_force_off_grid():
    """Eq. 3 and its adjoint written out term by term in pure Python (cmath, one loop per
    index), independent of the C library and of numpy's vectorisation, at arbitrary off-grid
    uv on a tiny window (nb = 8, 50 visibilities, odd and even offsets from the origin)."""
    import cmath
    rng = np.random.default_rng(12)
    nb, cell, m = 8, 7e-5, 50
    f = rng.standard_normal((nb, nb))
    u, v = rng.uniform(-9e3, 9e3, m), rng.uniform(-9e3, 9e3, m)
    c = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    fwd = []
    for j in range(m):
        acc = 0j
        for q in range(nb):
            for p in range(nb):
                l, mm = (p - nb // 2) * cell, (q - nb // 2) * cell
                acc += f[q, p] * cmath.exp(-2j * cmath.pi * (u[j] * l + v[j] * mm))
        fwd.append(acc)
    adj = np.zeros((nb, nb), complex)
    for q in range(nb):
        for p in range(nb):
            l, mm = (p - nb // 2) * cell, (q - nb // 2) * cell
            adj[q, p] = sum(c[j] * cmath.exp(2j * cmath.pi * (u[j] * l + v[j] * mm)) for j in range(m))
    got_f = oracle.model_vis(f, cell, u, v)
    got_a = oracle.adjoint(c, nb, cell, u, v)
    assert np.max(np.abs(got_f - np.array(fwd))) <= 1e-12 * np.max(np.abs(fwd))
    assert np.max(np.abs(got_a - adj)) <= 1e-12 * np.max(np.abs(adj))


# ------------------------------------------------------------------------------ adjoint
def test_adjoint_identity():
    rng = np.random.default_rng(5)
    nb, cell = 20, 3e-5
    x = rng.standard_normal((nb, nb))
    m = 300
    u, v = rng.uniform(-2e4, 2e4, m), rng.uniform(-2e4, 2e4, m)
    y = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    lhs = np.vdot(y, oracle.model_vis(x, cell, u, v)).real
    rhs = np.sum(x * oracle.adjoint(y, nb, cell, u, v).real)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10


def test_adjoint_on_grid_points_equals_ifft2():
    """Adjoint at grid-aligned points is nb^2 * ifft2 of the accumulated coefficients."""
    rng = np.random.default_rng(6)
    nb, cell = 16, 1e-4
    m = 80
    a = rng.integers(-30, 30, m)
    b = rng.integers(-30, 30, m)
    c = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    got = oracle.adjoint(c, nb, cell, a / (nb * cell), b / (nb * cell))
    G = np.zeros((nb, nb), complex)
    np.add.at(G, (b % nb, a % nb), c * np.exp(-1j * np.pi * (a + b)))
    expect = nb * nb * np.fft.ifft2(G)
    assert np.max(np.abs(got - expect)) <= 1e-10 * np.max(np.abs(expect))


def test_adjoint_pixels_match_full_window():
    rng = np.random.default_rng(7)
    nb, cell, m = 12, 4e-5, 90
    u, v = rng.uniform(-2e4, 2e4, m), rng.uniform(-2e4, 2e4, m)
    c = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    full = oracle.adjoint(c, nb, cell, u, v)
    qs, ps = rng.integers(0, nb, 20), rng.integers(0, nb, 20)
    assert np.allclose(oracle.adjoint_pixels(c, nb, cell, u, v, qs, ps), full[qs, ps], atol=1e-12)


# ----------------------------------------------------------------- windows and data term
def test_window_is_transpose_of_window_adjoint():
    rng = np.random.default_rng(8)
    img = rng.standard_normal((30, 30))
    win = rng.standard_normal((16, 16))
    for cx, cy in [(15, 15), (2, 28), (29, 0)]:
        lhs = np.sum(oracle.window(img, cx, cy, 16) * win)
        rhs = np.sum(img * oracle.window_adjoint(win, cx, cy, img.shape))
        assert abs(lhs - rhs) < 1e-12
    # pixel origin: window centre pixel nb/2 is the sky pixel (cy, cx)
    assert oracle.window(img, 7, 9, 16)[8, 8] == img[9, 7]


def _with_data(prob, sky=None, noise=True):
    sky = prob.sky_true if sky is None else sky
    for pair in prob.pairs:
        v = oracle.pair_model_vis(prob, sky, pair)
        if noise:
            v = v + pair.noise
        pair.vis = v.astype(np.complex64)
    return prob


def test_cost_zero_at_truth_without_noise():
    prob = _with_data(synth.small_mosaic(11, n=48, nb=32, nchan=2, npoint=2, ndump=3, n_ant=8),
                      noise=False)
    Q, g = oracle.data_cost_grad(prob, prob.sky_true)
    # complex64 rounding of V leaves a residual of ~1e-7 relative
    scale = sum(0.5 * float(np.sum(p.weight * np.abs(p.vis) ** 2)) for p in prob.pairs)
    assert Q <= 1e-12 * scale
    Qn, gn = oracle.data_cost_grad(prob, 1.1 * prob.sky_true)
    assert np.abs(g).max() <= 1e-3 * np.abs(gn).max()


def test_data_cost_is_weighted_half_square():
    """J = 1/2 sum w |r|^2: doubling every weight doubles Q; a unit-weight single visibility
    of a phase-centre source gives 1/2 |S - V|^2."""
    prob = _with_data(synth.small_mosaic(12, n=40, nb=32, nchan=1, npoint=1, ndump=3, n_ant=6))
    sky = prob.sky_true * 0.7
    Q1, _ = oracle.data_cost_grad(prob, sky)
    for p in prob.pairs:
        p.weight = p.weight * 2
    Q2, _ = oracle.data_cost_grad(prob, sky)
    assert abs(Q2 - 2 * Q1) <= 1e-10 * Q1
    one = synth.small_mosaic(13, n=16, nb=16, nchan=1, npoint=1, ndump=1, n_ant=2)
    one.centres[:] = [8, 8]
    one.beams[:] = 1.0
    one.pairs[0].uvw = one.pairs[0].uvw[:1]
    one.pairs[0].weight = np.ones(1, np.float32)
    one.pairs[0].vis = np.array([0.5 + 0.25j], np.complex64)
    s = np.zeros((1, 16, 16))
    s[0, 8, 8] = 2.0
    Q, _ = oracle.data_cost_grad(one, s)
    assert abs(Q - 0.5 * abs(2.0 - (0.5 + 0.25j)) ** 2) < 1e-12


def _fd_check(fun, x, idxs, h):
    f0, g = fun(x)
    for i in idxs:
        e = np.zeros_like(x)
        e.flat[i] = h
        fp, _ = fun(x + e)
        fm, _ = fun(x - e)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g.flat[i]) <= 1e-6 * max(abs(g).max(), 1e-30) + 1e-7 * abs(fd), (i, fd, g.flat[i])


def test_data_gradient_central_differences():
    prob = _with_data(synth.small_mosaic(14, n=40, nb=32, nchan=2, npoint=3, ndump=3, n_ant=7))
    rng = np.random.default_rng(14)
    x = prob.sky_true * rng.uniform(0.5, 1.5, prob.sky_true.shape)
    # pick pixels inside at least one window and some outside all windows
    idxs = rng.choice(x.size, 20, replace=False)
    _fd_check(lambda z: oracle.data_cost_grad(prob, z), x, idxs, 1e-4 * np.abs(x).max())


def test_data_grad_pixels_matches_full_gradient():
    prob = _with_data(synth.small_mosaic(15, n=40, nb=32, nchan=2, npoint=2, ndump=3, n_ant=7))
    x = prob.sky_true * 0.9
    _, g = oracle.data_cost_grad(prob, x)
    rng = np.random.default_rng(15)
    ys, xs = rng.integers(0, 40, 25), rng.integers(0, 40, 25)
    got = oracle.data_grad_pixels(prob, x, 1, ys, xs)
    assert np.allclose(got, g[1, ys, xs], rtol=1e-10, atol=1e-12 * np.abs(g).max())


# ------------------------------------------------------------------- regulariser (Eqs. 7-8)
def test_laplacian_kernel_is_the_papers():
    d, _ = _load_golden("laplacian_kernel.txt")
    assert np.array_equal(oracle.LAPLACIAN_KERNEL, d)
    img = np.zeros((9, 9))
    img[4, 4] = 1.0
    assert np.array_equal(oracle.laplacian(img)[3:6, 3:6], d)


def test_laplacian_matches_scipy_with_zero_boundary():
    rng = np.random.default_rng(16)
    img = rng.standard_normal((13, 17))
    d, _ = _load_golden("laplacian_kernel.txt")
    ref = scipy.ndimage.convolve(img, d, mode="constant", cval=0.0)
    assert np.allclose(oracle.laplacian(img), ref, atol=1e-13)


def test_regulariser_impulse_and_constant():
    stencil, meta = _load_golden("laplacian_impulse_gradient.txt")
    img = np.zeros((1, 11, 11))
    img[0, 5, 5] = 1.0
    R, g = oracle.reg_cost_grad(img)
    assert R == meta["R_at_impulse"]
    assert np.array_equal(g[0, 3:8, 3:8], stencil)
    assert np.count_nonzero(g) == np.count_nonzero(stencil)
    const = np.full((1, 12, 12), 3.0)
    R, g = oracle.reg_cost_grad(const)
    assert np.all(g[0, 2:-2, 2:-2] == 0.0)
    # boundary: zero padding makes the edge pixels' D I non-zero: sides 3, corners 6
    di = oracle.laplacian(const[0])
    assert di[0, 5] == 3.0 and di[0, 0] == 6.0 and di[5, 5] == 0.0


def test_regulariser_gradient_central_differences():
    rng = np.random.default_rng(17)
    x = rng.standard_normal((2, 10, 12))
    _fd_check(oracle.reg_cost_grad, x, rng.choice(x.size, 15, replace=False), 1e-4)


# ------------------------------------------------------------------- fusion term (Eqs. 11-13)
def test_dish_kernel_half_maximum_and_truncation():
    for fwhm in (4.0, 13.7, 58.0):
        b = oracle.dish_kernel(fwhm)
        r = (b.size - 1) // 2
        s = fwhm / (2 * math.sqrt(2 * math.log(2)))
        assert r == math.ceil(4 * s)
        assert abs(b.sum() - 1.0) < 1e-14
        # Gaussian value at +-FWHM/2 is half the peak (interpolate the continuous form)
        t = np.arange(-r, r + 1)
        peak = b[r]
        assert np.allclose(b, peak * np.exp(-0.5 * (t / s) ** 2), rtol=1e-12)
        assert abs(peak * math.exp(-0.5 * (fwhm / 2 / s) ** 2) - peak / 2) < 1e-12


def test_dish_conv_matches_scipy_convolve2d():
    rng = np.random.default_rng(18)
    img = rng.standard_normal((40, 33))
    b = oracle.dish_kernel(5.0)
    ref = scipy.signal.convolve2d(img, np.outer(b, b), mode="same", boundary="fill")
    assert np.allclose(oracle.dish_conv(img, b), ref, atol=1e-12)


def test_dish_conv_preserves_flux_away_from_edges():
    img = np.zeros((64, 64))
    img[30, 33] = 2.0
    b = oracle.dish_kernel(6.0)
    out = oracle.dish_conv(img, b)
    r = (b.size - 1) // 2
    assert abs(out.sum() - 2.0) < 1e-12
    assert np.allclose(out[30 - r:30 + r + 1, 33 - r:33 + r + 1], 2.0 * np.outer(b, b))


def test_fusion_zero_at_consistent_map_and_gradient():
    rng = np.random.default_rng(19)
    x = rng.uniform(0, 1, (2, 24, 20))
    b = oracle.dish_kernel(4.0)
    tsd = np.stack([oracle.dish_conv(x[c], b) for c in range(2)])
    K, g = oracle.fusion_cost_grad(x, tsd, [0.1, 0.2], 4.0)
    assert K < 1e-25 and np.abs(g).max() < 1e-10
    tsd2 = tsd + rng.standard_normal(tsd.shape) * 0.05
    _fd_check(lambda z: oracle.fusion_cost_grad(z, tsd2, [0.1, 0.2], 4.0), x,
              rng.choice(x.size, 15, replace=False), 1e-4)


# --------------------------------------------------------------------------- total (Eq. 14)
def test_total_cost_is_weighted_sum_of_terms():
    prob = _with_data(synth.small_mosaic(20, n=36, nb=32, nchan=1, npoint=2, ndump=3, n_ant=6,
                                         lambda_r=0.3, lambda_s=0.7, sd_fwhm_pix=4.0))
    b = oracle.dish_kernel(prob.sd_fwhm_pix)
    tsd = np.stack([oracle.dish_conv(prob.sky_true[c], b) for c in range(prob.nchan)])
    x = prob.sky_true * 0.8
    f, g, (Q, K, R) = oracle.cost_grad(prob, x, tsd, 0.05, with_terms=True)
    assert abs(f - (Q + 0.7 * K + 0.3 * R)) <= 1e-12 * f
    _fd_check(lambda z: oracle.cost_grad(prob, z, tsd, 0.05), x,
              np.random.default_rng(20).choice(x.size, 12, replace=False), 1e-4 * x.max())


# ----------------------------------------------------------------------------- solver (Eq. 10)
def test_solver_reaches_nnls_solution_of_tiny_problem():
    """With lambda = 0 the bounded problem is a non-negative least-squares fit; its unique
    solution (more visibilities than pixels) comes from scipy's NNLS on the explicit matrix."""
    prob = synth.small_mosaic(21, n=8, nb=8, nchan=1, npoint=1, ndump=16, n_ant=8,
                              lambda_r=0.0, lambda_s=0.0, sky_kind="points")
    prob.centres[:] = [4, 4]
    prob.sky_true = np.abs(np.random.default_rng(21).standard_normal((1, 8, 8)))
    prob.sky_true[0, :2] = 0.0  # part of the answer sits on the bound of Eq. 10
    _with_data(prob)
    pair = prob.pairs[0]
    cols = []
    for i in range(64):
        e = np.zeros((1, 8, 8))
        e.flat[i] = 1.0
        cols.append(oracle.pair_model_vis(prob, e, pair))
    A = np.array(cols).T
    sw = np.sqrt(pair.weight.astype(np.float64))
    M = np.concatenate([sw[:, None] * A.real, sw[:, None] * A.imag])
    y = np.concatenate([sw * pair.vis.real, sw * pair.vis.imag]).astype(np.float64)
    x_ref, _ = scipy.optimize.nnls(M, y, maxiter=10000)
    x, f, nit, nfev = oracle.solve_lbfgsb(prob, maxiter=500, pgtol=1e-12, factr=10.0)
    f_ref = 0.5 * np.sum((M @ x_ref - y) ** 2)
    assert f <= f_ref * (1 + 1e-6) + 1e-12
    assert np.linalg.cond(M) < 1e4
    assert np.allclose(x.ravel(), x_ref, atol=1e-3 * x_ref.max())
    assert np.count_nonzero(x_ref == 0.0) >= 4  # the bound is active: the pin tests it


def test_solver_point_source_flux_recovery():
    """Sect. 4.1: with lambda_r = lambda_s = 0 and positivity the flux of an unresolved source
    is recovered, and it collects in a single pixel. Criterion (ours, the paper prints no
    number): after 30 iterations each source pixel holds its input flux within 1 %, on a
    C1-shaped problem (36 antennas, 13 dumps over +-5 h, 1 mJy noise) with a 64^2 sky."""
    rng = synth.make_rng(1001)
    n = 64
    cell = 8.0 * synth.ARCSEC
    enu = synth.antenna_layout(rng, 36, 6000.0)
    ha = np.linspace(-5, 5, 13) * 15 * synth.DEG
    uvw = synth.uvw_tracks(enu, ha, synth.DEC_LMC_RAD, synth.LAT_ASKAP_RAD, synth.HI_FREQ_HZ)
    sky = synth.point_source_sky(rng, n, 5, 8, 56, 0.1, 1.0)[None]
    beam = synth.gaussian_beam(n, synth.DEG / cell).astype(np.float32)[None]
    pair = synth.VisSet(0, 0, uvw.astype(np.float32), np.full(uvw.shape[0], 1e6, np.float32),
                        synth.complex_noise(rng, uvw.shape[0], 1e-3))
    prob = synth.Problem("c1_lite", n, cell, 1, n, np.array([[n // 2, n // 2]]), beam, [pair],
                         sky, positivity=True)
    _with_data(prob)
    x, f, nit, nfev = oracle.solve_lbfgsb(prob, maxiter=30)
    ys, xs = np.nonzero(sky[0])
    for yy, xx in zip(ys, xs):
        assert abs(x[0, yy, xx] - sky[0, yy, xx]) <= 0.01 * sky[0, yy, xx], (yy, xx)
    assert x.min() >= 0.0
    # the bounded problem's optimality: the projected gradient is far below the initial one
    _, g0 = oracle.cost_grad(prob, np.zeros_like(x))
    _, g = oracle.cost_grad(prob, x)
    pg = np.abs(np.maximum(x - g, 0.0) - x).max()
    assert pg < 1e-2 * np.abs(g0).max()


def test_regularisation_spreads_point_source_flux_over_adjacent_pixels():
    """Sect. 4.1: a regulariser moves an unresolved source's flux from its pixel to the adjacent
    ones, so lambda_r = 0 is the setting for point-source photometry. Same problem as the
    flux-recovery pin: with lambda_r = 0 each source pixel holds its flux within 1 %; with a
    Laplacian strong enough to matter (lambda_r = 1e8, against sum w = 8.2e9 per pixel) every
    source pixel loses more than 10 % and its eight neighbours gain."""
    rng = synth.make_rng(1001)
    n = 64
    cell = 8.0 * synth.ARCSEC
    enu = synth.antenna_layout(rng, 36, 6000.0)
    ha = np.linspace(-5, 5, 13) * 15 * synth.DEG
    uvw = synth.uvw_tracks(enu, ha, synth.DEC_LMC_RAD, synth.LAT_ASKAP_RAD, synth.HI_FREQ_HZ)
    sky = synth.point_source_sky(rng, n, 5, 8, 56, 0.1, 1.0)[None]
    beam = synth.gaussian_beam(n, synth.DEG / cell).astype(np.float32)[None]
    pair = synth.VisSet(0, 0, uvw.astype(np.float32), np.full(uvw.shape[0], 1e6, np.float32),
                        synth.complex_noise(rng, uvw.shape[0], 1e-3))
    ys, xs = np.nonzero(sky[0])
    peak, ring = {}, {}
    for lr in (0.0, 1e8):
        prob = synth.Problem("c1_lite", n, cell, 1, n, np.array([[n // 2, n // 2]]), beam, [pair], sky,
                             lambda_r=lr, positivity=True)
        _with_data(prob)
        x, *_ = oracle.solve_lbfgsb(prob, maxiter=30)
        peak[lr] = x[0][ys, xs] / sky[0][ys, xs]
        ring[lr] = np.array([x[0][y - 1:y + 2, c - 1:c + 2].sum() - x[0][y, c] for y, c in zip(ys, xs)])
    assert np.all(np.abs(peak[0.0] - 1.0) <= 0.01), peak[0.0]
    assert np.all(peak[1e8] < 0.9), peak[1e8]
    assert np.all(ring[1e8] > ring[0.0] + 0.05 * sky[0][ys, xs]), (ring[0.0], ring[1e8])


def test_point_source_spectrum_fixture_matches_stated_law():
    rows, meta = _load_golden("point_source_spectrum.txt")
    assert rows.shape == (10, 2) and meta["noise_jy"] == 0.1
    assert np.allclose(synth.point_source_flux_law(rows[:, 0]), rows[:, 1], rtol=1e-14)
    assert np.isclose(rows[:, 0].mean(), 1.0e9) and np.allclose(np.diff(rows[:, 0]), 0.1e9)


def test_point_source_spectrum_recovered_per_channel():
    """Sect. 4.1, multi-frequency: ten channels of a point source with S = 5 (nu/1.5 GHz)^-1
    at the phase centre, 0.1 Jy noise, lambda_r = lambda_s = 0, positivity: the flux of each
    channel collects in the source pixel, within 3x its noise-propagated error. That error is
    the least-squares one of a single flux at the phase centre (beam 1 there) from M_c complex
    samples with sigma per component: sigma / sqrt(M_c). A channel that borrowed another
    channel's data, beam or sky plane would miss by 6 % or more (adjacent fluxes differ so)."""
    rows, meta = _load_golden("point_source_spectrum.txt")
    prob = _with_data(synth.point_source_spectrum(sigma=meta["noise_jy"]))
    n = prob.n
    assert np.allclose(prob.freqs_hz, rows[:, 0], rtol=0) and prob.nchan == 10
    assert np.allclose(prob.sky_true[:, n // 2, n // 2], rows[:, 1], rtol=1e-14)
    x, f, nit, nfev = oracle.solve_lbfgsb(prob, maxiter=30)
    assert x.min() >= 0.0
    m = np.array([p.m for p in sorted(prob.pairs, key=lambda p: p.chan)])
    err = x[:, n // 2, n // 2] - rows[:, 1]
    assert np.all(np.abs(err) <= 3.0 * meta["noise_jy"] / np.sqrt(m)), err * np.sqrt(m) / meta["noise_jy"]
    # the recovered spectrum has the input's index
    alpha = np.polyfit(np.log(rows[:, 0]), np.log(x[:, n // 2, n // 2]), 1)[0]
    assert abs(alpha + 1.0) <= 1e-3, alpha


def _radial_band_power(img, k_lo, k_hi):
    """Mean |FFT|^2 over integer radial frequencies k_lo <= |k| < k_hi (cycles per field)."""
    n = img.shape[-1]
    k = np.hypot(np.fft.fftfreq(n)[:, None], np.fft.fftfreq(n)[None, :]) * n
    return float(np.mean(np.abs(np.fft.fft2(img))[(k >= k_lo) & (k < k_hi)] ** 2))


def test_regularisation_strength_suppresses_noise_and_high_frequencies():
    """Sect. 4.2 (noise-only observation): as lambda_r grows through 0, 0.1, 1, 10, 100 the
    reconstruction's noise level falls and its high spatial frequencies are progressively
    suppressed. Single pointing, noise-only visibilities (5 Jy per component), a compact
    24-antenna array sampled below the pixel Nyquist limit, no positivity bound (noise is
    signed)."""
    n, cell = 32, 3.0 * synth.ARCSEC
    rng = synth.make_rng(1020)
    enu = synth.antenna_layout(rng, 24, 8000.0)
    ha = (np.arange(12) + 0.5 - 6) * (3000.0 / 86400.0) * 2 * np.pi
    uvw = synth.uvw_tracks(enu, ha, -69.04 * synth.DEG, -30.7 * synth.DEG, synth.HI_FREQ_HZ)
    assert np.abs(uvw[:, :2]).max() < 0.5 / cell
    m, sig = uvw.shape[0], 5.0
    pair = synth.VisSet(0, 0, uvw.astype(np.float32), np.full(m, 1 / sig ** 2, np.float32),
                        synth.complex_noise(rng, m, sig))
    beam = synth.gaussian_beam(n, synth.DEG / cell).astype(np.float32)[None]
    var, high = [], []
    for lr in (0.0, 0.1, 1.0, 10.0, 100.0):
        prob = synth.Problem("noise_only", n, cell, 1, n, np.array([[n // 2, n // 2]]), beam, [pair],
                             np.zeros((1, n, n)), lambda_r=lr, positivity=False)
        _with_data(prob)
        x, *_ = oracle.solve_lbfgsb(prob, maxiter=50)
        var.append(float(x.var()))
        high.append(_radial_band_power(x[0], n / 4, n / 2))
    assert all(a > b for a, b in zip(var, var[1:])), var
    assert all(a > b for a, b in zip(high, high[1:])), high
    assert high[-1] < 1e-2 * high[0], high


def test_noise_grows_away_from_the_pointing_centre():
    """Sect. 4.2: with the primary beam in the forward model, the noise of a reconstruction
    from noise-only data grows away from the pointing centre, with and without the Laplacian
    (the beam, not the regulariser, drives it). A 12 px FWHM beam on a 32^2 field: the image's
    spread beyond one FWHM from the centre is more than 1.5 times that within half of it."""
    n, cell, fwhm = 32, 3.0 * synth.ARCSEC, 12.0
    rng = synth.make_rng(1020)
    enu = synth.antenna_layout(rng, 24, 8000.0)
    ha = (np.arange(12) + 0.5 - 6) * (3000.0 / 86400.0) * 2 * np.pi
    uvw = synth.uvw_tracks(enu, ha, -69.04 * synth.DEG, -30.7 * synth.DEG, synth.HI_FREQ_HZ)
    m, sig = uvw.shape[0], 5.0
    pair = synth.VisSet(0, 0, uvw.astype(np.float32), np.full(m, 1 / sig ** 2, np.float32),
                        synth.complex_noise(rng, m, sig))
    beam = synth.gaussian_beam(n, fwhm).astype(np.float32)[None]
    yy, xx = np.indices((n, n)) - n // 2
    r = np.hypot(yy, xx)
    for lr in (0.0, 1.0):
        prob = synth.Problem("noise_only_beam", n, cell, 1, n, np.array([[n // 2, n // 2]]), beam, [pair],
                             np.zeros((1, n, n)), lambda_r=lr, positivity=False)
        _with_data(prob)
        x, *_ = oracle.solve_lbfgsb(prob, maxiter=50)
        inner, outer = x[0][r < fwhm / 2].std(), x[0][(r > fwhm) & (r < n / 2)].std()
        assert outer > 1.5 * inner, (lr, inner, outer)


def test_fusion_restores_the_large_scales_the_interferometer_misses():
    """Sect. 2.4 and 4.3: the interferometer cannot see the lowest spatial frequencies (here no
    baseline shorter than 3 cycles per field, and never k = 0); fused with a single-dish map of
    the same sky (lambda_s = 1, 5 % noise) the reconstruction recovers them. Lognormal sky,
    single pointing, positivity, no Laplacian: without fusion the k < 3 part of the image
    misses by tens of per cent and the total flux by about a fifth; with fusion both come
    within a few per cent."""
    n, cell = 32, 20.0 * synth.ARCSEC
    rng = synth.make_rng(1030)
    enu = synth.antenna_layout(rng, 24, 1000.0)
    ha = (np.arange(12) + 0.5 - 6) * (3000.0 / 86400.0) * 2 * np.pi
    uvw = synth.uvw_tracks(enu, ha, synth.DEC_LMC_RAD, synth.LAT_ASKAP_RAD, synth.HI_FREQ_HZ)
    k_uv = np.hypot(uvw[:, 0], uvw[:, 1]) * n * cell
    assert k_uv.max() < n / 2
    uvw = uvw[k_uv >= 3.0]
    m, sig = uvw.shape[0], 1e-3
    pair = synth.VisSet(0, 0, uvw.astype(np.float32), np.full(m, 1 / sig ** 2, np.float32),
                        synth.complex_noise(rng, m, sig))
    sky = synth.lognormal_sky(rng, n)[None]
    beam = synth.gaussian_beam(n, synth.DEG / cell).astype(np.float32)[None]

    def low_k(img):
        F = np.fft.fft2(img)
        F[np.hypot(np.fft.fftfreq(n)[:, None], np.fft.fftfreq(n)[None, :]) * n >= 3.0] = 0.0
        return np.fft.ifft2(F).real

    err = {}
    for ls in (0.0, 1.0):
        prob = synth.Problem("fusion", n, cell, 1, n, np.array([[n // 2, n // 2]]), beam, [pair], sky,
                             lambda_r=0.0, lambda_s=ls, positivity=True, sd_fwhm_pix=4.0,
                             sd_noise_unit=synth.make_rng(5).standard_normal((1, n, n)))
        attach_data(prob)
        kw = dict(tsd=prob.tsd, sigma_sd=prob.sigma_sd) if ls > 0 else {}
        x, *_ = oracle.solve_lbfgsb(prob, maxiter=60, **kw)
        err[ls] = (np.linalg.norm(low_k(x[0]) - low_k(sky[0])) / np.linalg.norm(low_k(sky[0])),
                   abs(x.sum() - sky.sum()) / sky.sum())
    assert err[0.0][0] > 0.1 and err[0.0][1] > 0.1, err
    assert err[1.0][0] < 0.05 and err[1.0][1] < 0.01, err
    assert err[1.0][0] < 0.1 * err[0.0][0], err


def test_joint_deconvolution_recovers_more_large_scale_structure_than_linear_mosaicking():
    """Sect. 4.3: jointly deconvolving all pointings of a mosaic recovers the large scales
    better than mosaicking independently deconvolved pointings. Seven pointings (hexagonal,
    pitch 12 px, Gaussian beams of 12 px FWHM on 32 px windows) over a 48^2 lognormal sky,
    no baseline below 3 cycles per window, positivity, no regularisation, 60 iterations each.
    Linear mosaic (our reading; the paper prints no weights): sum_k A_k^2 x_k / sum_k A_k^2,
    x_k the pointing's own solve. Inside the effective-beam mask (sum_k A_k^2 >= 0.2 of its
    peak, as in the paper's figure) the k < 4 part of the joint image is closer to the truth
    by more than a factor two."""
    n, nb = 48, 32
    cell = 20.0 * synth.ARCSEC
    rng = synth.make_rng(1040)
    enu = synth.antenna_layout(rng, 24, 1000.0)
    ha = (np.arange(12) + 0.5 - 6) * (3000.0 / 86400.0) * 2 * np.pi
    uvw = synth.uvw_tracks(enu, ha, synth.DEC_LMC_RAD, synth.LAT_ASKAP_RAD, synth.HI_FREQ_HZ)
    k_uv = np.hypot(uvw[:, 0], uvw[:, 1]) * nb * cell
    assert k_uv.max() < nb / 2
    uvw = uvw[k_uv >= 3.0].astype(np.float32)
    centres = np.array([[12, 24], [24, 24], [36, 24], [18, 14], [30, 14], [18, 34], [30, 34]])
    sky = synth.lognormal_sky(rng, n)[None]
    beam = synth.gaussian_beam(nb, 12.0).astype(np.float32)
    beams = np.stack([beam] * len(centres))
    m, sig = uvw.shape[0], 1e-3
    pairs = [synth.VisSet(k, 0, uvw, np.full(m, 1 / sig ** 2, np.float32), synth.complex_noise(rng, m, sig))
             for k in range(len(centres))]
    prob = synth.Problem("mosaic", n, cell, 1, nb, centres, beams, pairs, sky, positivity=True)
    attach_data(prob)
    x_joint, *_ = oracle.solve_lbfgsb(prob, maxiter=60)
    num, den = np.zeros((n, n)), np.zeros((n, n))
    for k, pair in enumerate(pairs):
        one = synth.Problem("pointing", n, cell, 1, nb, centres[k:k + 1], beams[k:k + 1],
                            [synth.VisSet(0, 0, pair.uvw, pair.weight, pair.noise, pair.vis)], sky,
                            positivity=True)
        xk, *_ = oracle.solve_lbfgsb(one, maxiter=60)
        a2 = oracle.window_adjoint(beam.astype(np.float64) ** 2, int(centres[k][0]), int(centres[k][1]), (n, n))
        num += a2 * xk[0]
        den += a2
    x_lin = num / np.maximum(den, 1e-30)
    mask = den >= 0.2 * den.max()
    kk = np.hypot(np.fft.fftfreq(n)[:, None], np.fft.fftfreq(n)[None, :]) * n

    def low_k_error(img):
        F = np.fft.fft2((img - sky[0]) * mask)
        F0 = np.fft.fft2(sky[0] * mask)
        return np.linalg.norm(F[kk < 4]) / np.linalg.norm(F0[kk < 4])

    e_joint, e_lin = low_k_error(x_joint[0]), low_k_error(x_lin)
    assert e_joint < 0.5 * e_lin, (e_joint, e_lin)


# ------------------------------------------------------- SIN re-projection grids (Eq. 2)
def test_bilinear_on_integer_grid_is_the_window():
    rng = np.random.default_rng(30)
    img = rng.standard_normal((40, 36))
    for cx, cy in [(18, 20), (2, 35), (39, 1)]:
        g = synth.projection_grid(16, cx, cy)
        assert np.array_equal(oracle.bilinear(img, g), oracle.window(img, cx, cy, 16))


def test_bilinear_reproduces_linear_functions_and_matches_scipy():
    ny, nx = 30, 34
    Y, X = np.mgrid[0:ny, 0:nx]
    img = 0.5 + 0.25 * X - 0.75 * Y
    g = synth.projection_grid(12, 16.3, 14.7, rot_rad=0.3, scale=1.1, curvature=0.05)
    got = oracle.bilinear(img, g)
    expect = 0.5 + 0.25 * g[..., 0].astype(np.float64) - 0.75 * g[..., 1].astype(np.float64)
    assert np.allclose(got, expect, atol=1e-12)
    rng = np.random.default_rng(31)
    img = rng.standard_normal((ny, nx))
    ref = scipy.ndimage.map_coordinates(img, [g[..., 1].astype(np.float64), g[..., 0].astype(np.float64)],
                                        order=1, mode="constant", cval=0.0)
    assert np.allclose(oracle.bilinear(img, g), ref, atol=1e-12)


def test_bilinear_adjoint_identity_with_edges_and_nan():
    rng = np.random.default_rng(32)
    img = rng.standard_normal((20, 22))
    g = synth.projection_grid(16, 3.4, 18.8, rot_rad=-0.5, scale=1.3)
    g[0, 0] = np.nan
    win = rng.standard_normal((16, 16))
    lhs = np.sum(oracle.bilinear(img, g) * win)
    rhs = np.sum(img * oracle.bilinear_adjoint(win, g, img.shape))
    assert abs(lhs - rhs) < 1e-12 and oracle.bilinear(img, g)[0, 0] == 0.0


def test_gridded_data_gradient_central_differences():
    prob = synth.small_mosaic(33, n=40, nb=32, nchan=1, npoint=2, ndump=3, n_ant=7)
    prob.grids = {0: synth.projection_grid(32, 20.4, 19.6, rot_rad=0.2, scale=0.9, curvature=0.03)}
    _with_data(prob)
    rng = np.random.default_rng(33)
    x = prob.sky_true * rng.uniform(0.5, 1.5, prob.sky_true.shape)
    _fd_check(lambda z: oracle.data_cost_grad(prob, z), x, rng.choice(x.size, 15, replace=False),
              1e-4 * np.abs(x).max())



def test_sampled_data_gradient_refuses_reprojected_pointings():
    """The sampled gradient follows integer windows only; with a re-projection grid (Eq. 2) it
    raises rather than answer with the wrong window, and pointings without a grid still work."""
    prob = synth.small_mosaic(34, n=40, nb=32, nchan=1, npoint=2, ndump=3, n_ant=7)
    prob.grids = {1: synth.projection_grid(32, 20.4, 19.6, rot_rad=0.2, scale=0.9)}
    _with_data(prob)
    x = prob.sky_true * 0.5
    with pytest.raises(NotImplementedError):
        oracle.data_grad_pixels(prob, x, 0, [10, 20], [11, 21])
    prob.grids = {}
    _with_data(prob)
    _, g = oracle.data_cost_grad(prob, x)
    assert np.allclose(oracle.data_grad_pixels(prob, x, 0, [10, 20], [11, 21]), g[0, [10, 20], [11, 21]],
                       rtol=1e-10, atol=1e-12 * np.abs(g).max())


# ------------------------------------------------- Toeplitz form of the data term (Eqs. 3-6)
def test_psf_kernel_centre_symmetry_and_normal_matrix():
    """T(0) = sum w; T(-d) = conj T(d); and on a tiny window the explicit normal matrix
    F^H W F (built column by column from the forward DFT) has entries T(p - q)."""
    prob = _with_data(synth.small_mosaic(41, n=24, nb=8, nchan=1, npoint=1, ndump=3, n_ant=5,
                                         lambda_r=0.0, lambda_s=0.0))
    pair = prob.pairs[0]
    nb = prob.nb
    T = oracle.psf_kernel(pair, nb, prob.cell_rad)
    w = pair.weight.astype(np.float64)
    assert abs(T[nb, nb] - w.sum()) <= 1e-12 * w.sum()
    for dy, dx in [(1, 2), (-3, 5), (7, -7), (0, -4)]:
        assert abs(T[nb - dy, nb - dx] - np.conj(T[nb + dy, nb + dx])) <= 1e-9 * w.sum()
    cols = []
    for i in range(nb * nb):
        e = np.zeros((nb, nb))
        e.flat[i] = 1.0
        cols.append(oracle.model_vis(e, prob.cell_rad, pair.uvw[:, 0], pair.uvw[:, 1]))
    F = np.array(cols).T                                  # [m][nb*nb]
    H = F.conj().T @ (w[:, None] * F)
    qy, qx = np.divmod(np.arange(nb * nb), nb)
    Tpq = T[nb + qy[:, None] - qy[None, :], nb + qx[:, None] - qx[None, :]]
    assert np.allclose(H, Tpq, rtol=0, atol=1e-9 * w.sum())


def test_toeplitz_data_term_equals_the_direct_one():
    """The expansion is exact: the Toeplitz cost and gradient equal the direct ones (Eqs. 5-6)
    to rounding, windows off the sky edge and ragged pairs included; a re-projected pointing
    too (the operator acts on the window)."""
    prob = _with_data(synth.small_mosaic(42, n=40, nb=16, nchan=2, npoint=3, ndump=4, n_ant=6,
                                         lambda_r=0.0, lambda_s=0.0))
    prob.grids = {1: synth.projection_grid(16, float(prob.centres[1][0]) + 0.3,
                                           float(prob.centres[1][1]) - 0.6, 0.2, 1.05, 0.02)}
    x = np.abs(np.random.default_rng(42).standard_normal(prob.sky_true.shape))
    Q, g = oracle.data_cost_grad(prob, x)
    Qt, gt = oracle.toeplitz_data_cost_grad(prob, x)
    assert abs(Qt - Q) <= 1e-11 * Q
    assert np.linalg.norm(gt - g) <= 1e-11 * np.linalg.norm(g)


def test_toeplitz_single_zero_spacing_closed_form():
    """One visibility at u = v = 0 (T = w everywhere): the model is the window sum, so
    Q = w/2 |sum z - V|^2 and dQ/dz = w (sum z - Re V) on every window pixel."""
    prob = synth.small_mosaic(43, n=16, nb=16, nchan=1, npoint=1, ndump=1, n_ant=2,
                              lambda_r=0.0, lambda_s=0.0)
    prob.centres[:] = [8, 8]
    pair = prob.pairs[0]
    pair.uvw = np.zeros((1, 3), np.float32)
    pair.weight = np.array([2.5], np.float32)
    pair.vis = np.array([1.5 - 0.25j], np.complex64)
    x = np.random.default_rng(43).uniform(0, 1, (1, 16, 16))
    A = prob.beams[0].astype(np.float64)
    s = float(np.sum(A * x[0]))
    Q, g = oracle.toeplitz_data_cost_grad(prob, x)
    assert abs(Q - 0.5 * 2.5 * ((s - 1.5) ** 2 + 0.25 ** 2)) <= 1e-12 * Q
    assert np.allclose(g[0], A * 2.5 * (s - 1.5), rtol=1e-12, atol=0)


# ------------------------------------------------- feathering (short-spacing appendix)
def test_rayleigh_jeans_factor_matches_the_radio_rule_of_thumb():
    """T_B = 1.222e3 S / (nu^2 theta^2) (K, mJy per Gaussian beam, GHz, arcsec; the standard
    NRAO conversion) gives S / Omega for 1 K at 1.4204 GHz with Omega = pi theta^2 / (4 ln 2)."""
    nu_ghz, theta = 1.4204058, 7.0
    s_mjy = nu_ghz ** 2 * theta ** 2 / 1.222e3
    omega = math.pi * theta ** 2 / (4.0 * math.log(2.0))
    ref = s_mjy * 1e-3 / omega
    assert abs(oracle.rayleigh_jeans_factor(nu_ghz * 1e9) - ref) <= 1e-3 * ref


def test_feather_limits_and_identities():
    rng = np.random.default_rng(51)
    a = rng.standard_normal((2, 64, 64))
    b = rng.standard_normal((2, 64, 64))
    # identical maps are left unchanged
    assert np.allclose(oracle.feather(a, a, 9.0), a, atol=1e-12)
    # theta -> 0: B = 1 everywhere, the single-dish map
    assert np.allclose(oracle.feather(a, b, 1e-9), b, atol=1e-12)
    # theta -> infinity: only the k = 0 term of the single-dish map survives
    big = oracle.feather(a, b, 1e6)
    assert np.allclose(big, a + (b - a).mean(axis=(1, 2), keepdims=True), atol=1e-10)
    # the scale multiplies the single-dish map
    assert np.allclose(oracle.feather(a, b, 5.0, 2.5), oracle.feather(a, 2.5 * b, 5.0), atol=1e-12)


def test_feather_of_an_impulse_is_the_gaussian_of_the_transfer_function():
    """Interferometric map zero, single-dish map a unit impulse: the result is the inverse
    transform of B, a unit-area Gaussian of sigma = theta / (2 sqrt(2 ln 2)) pixels (its
    periodic copies are negligible for sigma << n)."""
    n, theta = 128, 12.0
    sd = np.zeros((1, n, n))
    sd[0, 0, 0] = 1.0
    out = oracle.feather(np.zeros((1, n, n)), sd, theta)[0]
    sig = theta / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    d = np.minimum(np.arange(n), n - np.arange(n))
    g = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * sig ** 2)) / (2 * math.pi * sig ** 2)
    assert np.abs(out - g).max() <= 1e-12
    assert abs(out.sum() - 1.0) <= 1e-12


# ------------------------------------------------- full visibility equation (Eq. 1, w-term)
def test_wterm_phase_is_the_geometric_delay():
    """Eq. 1's phase u l + v m + w (n - 1) is the geometric delay difference b.(s - s0)/lambda
    between a source direction s and the phase centre s0, with b and s taken in the equatorial
    frame of the hour angle (independent of the (u, v, w) decomposition); the coplanar Eq. 3
    misses w (n - 1). Amplitude f / n."""
    lat, dec0, ha = synth.LAT_ASKAP_RAD, synth.DEC_LMC_RAD, 1.3
    enu = np.array([[0.0, 0.0, 0.0], [4200.0, -2500.0, 30.0]])
    uvw = synth.uvw_tracks(enu, np.array([ha]), dec0, lat, synth.HI_FREQ_HZ)
    lam = synth.C_LIGHT / synth.HI_FREQ_HZ
    b = enu[1] - enu[0]
    bxyz = np.array([-math.sin(lat) * b[1] + math.cos(lat) * b[2], b[0],
                     math.cos(lat) * b[1] + math.sin(lat) * b[2]]) / lam
    # phase centre and a source 25 and 19 pixels off it (1 arcmin cells), as unit vectors
    nb, cell = 64, 60.0 * synth.ARCSEC
    p, q = nb // 2 + 25, nb // 2 - 19
    l, m = (p - nb // 2) * cell, (q - nb // 2) * cell
    n = math.sqrt(1.0 - l * l - m * m)
    ch, sh, cd, sd = math.cos(ha), math.sin(ha), math.cos(dec0), math.sin(dec0)
    s0 = np.array([cd * ch, -cd * sh, sd])
    # tangent-plane axes at s0: east (increasing right ascension) and north
    e_l = np.array([sh, ch, 0.0])
    e_m = np.cross(s0, e_l)
    s = l * e_l + m * e_m + n * s0
    delay = float(bxyz @ (s - s0))
    f = np.zeros((nb, nb))
    f[q, p] = 2.0
    V = oracle.model_vis(f, cell, uvw[:, 0], uvw[:, 1], uvw[:, 2])[0]
    assert abs(abs(V) - 2.0 / n) <= 1e-12
    ph = -2.0 * math.pi * delay
    assert abs(V - 2.0 / n * complex(math.cos(ph), math.sin(ph))) <= 1e-9
    Vc = oracle.model_vis(f, cell, uvw[:, 0], uvw[:, 1])[0]
    assert abs(np.angle(V / Vc) - np.angle(np.exp(-2j * math.pi * uvw[0, 2] * (n - 1.0)))) <= 1e-9
    assert abs(uvw[0, 2] * (n - 1.0)) > 0.05  # the test geometry makes the w-term visible


def test_wterm_adjoint_identity_and_gradient():
    rng = np.random.default_rng(61)
    nb, cell, m = 24, 90.0 * synth.ARCSEC, 40
    uvw = rng.standard_normal((m, 3)) * np.array([3000.0, 3000.0, 8000.0])
    f = rng.standard_normal((nb, nb))
    c = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    Ff = oracle.model_vis(f, cell, uvw[:, 0], uvw[:, 1], uvw[:, 2])
    a = oracle.adjoint(c, nb, cell, uvw[:, 0], uvw[:, 1], uvw[:, 2])
    lhs = np.vdot(c, Ff)
    rhs = np.vdot(a, f.astype(complex))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    qs, ps = rng.integers(0, nb, 9), rng.integers(0, nb, 9)
    ap = oracle.adjoint_pixels(c, nb, cell, uvw[:, 0], uvw[:, 1], qs, ps, uvw[:, 2])
    assert np.allclose(ap, a[qs, ps], rtol=0, atol=1e-11 * np.abs(a).max())
    prob = synth.small_mosaic(62, n=40, nb=32, nchan=1, npoint=2, ndump=3, n_ant=7,
                              cell_arcsec=120.0, lambda_r=0.0, lambda_s=0.0)
    prob.wterm = True
    _with_data(prob)
    x = prob.sky_true * rng.uniform(0.5, 1.5, prob.sky_true.shape)
    _fd_check(lambda z: oracle.data_cost_grad(prob, z), x, rng.choice(x.size, 10, replace=False), 1e-4)
