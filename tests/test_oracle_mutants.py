"""The pins catch plausible mistakes: each case plants one mistake in the oracle (on the CPU,
by replacing one oracle function for the duration of the test) and checks that the pins aimed
at it fail. A pin that still passed with the mistake in place would not be pinning anything.
Every planted mistake changes what the method computes (conjugating the adjoint's output, for
instance, does not: only its real part enters the gradient; using the forward's exponent sign
in the adjoint does)."""
import math

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins


def _conj_forward(orig):
    return lambda f, cell, u, v, w=None: np.conj(orig(f, cell, u, v, w))


def _swap_uv(orig):
    return lambda f, cell, u, v, w=None: orig(f, cell, v, u, w)


def _origin_off_by_one(orig):
    return lambda f, cell, u, v, w=None: orig(np.roll(np.asarray(f, dtype=np.float64), 1, axis=1), cell, u, v, w)


def _adjoint_forward_sign(orig):
    # sum_j c_j exp(-2 pi i (u l + v m)): the forward's sign in the adjoint
    return lambda c, nb, cell, u, v, w=None: np.conj(orig(np.conj(np.asarray(c)), nb, cell, u, v, w))


def _no_half_in_j(orig):
    def f(prob, sky, with_grad=True):
        Q, g = orig(prob, sky, with_grad)
        return 2.0 * Q, g
    return f


def _fwhm_as_sigma(orig):
    return lambda fwhm: orig(fwhm * 2.0 * math.sqrt(2.0 * math.log(2.0)))


def _fusion_grad_without_inverse_variance(orig):
    def f(x, tsd, sigma_sd, fwhm):
        K, g = orig(x, tsd, sigma_sd, fwhm)
        return K, g * np.asarray(sigma_sd, dtype=np.float64)[:, None, None] ** 2
    return f


def _laplacian_centre_five(orig):
    return lambda img: orig(img) + np.asarray(img, dtype=np.float64)


def _window_transposed(orig):
    return lambda img, cx, cy, nb: orig(img, cx, cy, nb).T


def _bilinear_xy_exchanged(orig):
    return lambda img, grid: orig(img, np.ascontiguousarray(np.asarray(grid)[..., ::-1]))


def _w_sign(orig):
    return lambda f, cell, u, v, w=None: orig(f, cell, u, v, None if w is None else -np.asarray(w, dtype=np.float64))


def _psf_conjugated(orig):
    return lambda pair, nb, cell: np.conj(orig(pair, nb, cell))


def _feather_weights_exchanged(orig):
    # B applied to the interferometric map and 1 - B to the single-dish one
    return lambda i_int, i_sd, theta_pix, sd_scale=1.0: orig(np.asarray(i_sd) * sd_scale, np.asarray(i_int) / sd_scale,
                                                            theta_pix, sd_scale)


def _rj_twice(orig):
    return lambda freq_hz: 2.0 * orig(freq_hz)


def _laplacian_periodic(orig):
    def f(img):
        img = np.asarray(img, dtype=np.float64)
        return (4 * img - np.roll(img, 1, 0) - np.roll(img, -1, 0) - np.roll(img, 1, 1) - np.roll(img, -1, 1))
    return f


def _data_gradient_without_beam(orig):
    def f(prob, sky, with_grad=True):
        saved = prob.beams
        Q, _ = orig(prob, sky, with_grad=False)
        prob.beams = np.ones_like(saved)
        try:
            _, g = orig(prob, sky, with_grad)
        finally:
            prob.beams = saved
        return Q, g
    return f


def _w_without_inverse_n(orig):
    def f(img, cell, u, v, w=None):
        if w is None:
            return orig(img, cell, u, v)
        img = np.asarray(img, dtype=np.float64)
        c = (np.arange(img.shape[0]) - img.shape[0] // 2) * cell
        n = np.sqrt(1.0 - c[:, None] ** 2 - c[None, :] ** 2)
        return orig(img * n, cell, u, v, w)  # cancels the 1/n of Eq. 1
    return f


MUTANTS = [
    ("sign of the forward exponent", "model_vis", _conj_forward,
     [pins.test_forward_offset_source_phase_direction, pins.test_forward_on_grid_points_equals_fft2]),
    ("u and v exchanged (l, m transposed)", "model_vis", _swap_uv,
     [pins.test_forward_offset_source_phase_direction, pins.test_forward_and_adjoint_brute_force_off_grid]),
    ("pixel origin off by one", "model_vis", _origin_off_by_one,
     [pins.test_forward_phase_centre_source_is_flat, pins.test_forward_and_adjoint_brute_force_off_grid]),
    ("adjoint with the forward's exponent sign", "adjoint", _adjoint_forward_sign,
     [pins.test_adjoint_identity, pins.test_adjoint_on_grid_points_equals_ifft2]),
    ("the 1/2 of J dropped", "data_cost_grad", _no_half_in_j, [pins.test_data_cost_is_weighted_half_square]),
    ("dish FWHM used as sigma", "dish_kernel", _fwhm_as_sigma, [pins.test_dish_kernel_half_maximum_and_truncation]),
    ("fusion gradient without 1/sigma_sd^2", "fusion_cost_grad", _fusion_grad_without_inverse_variance,
     [pins.test_fusion_zero_at_consistent_map_and_gradient]),
    ("Laplacian centre weight 5", "laplacian", _laplacian_centre_five, [pins.test_regulariser_impulse_and_constant]),
    ("window transposed", "window", _window_transposed, [pins.test_bilinear_on_integer_grid_is_the_window]),
    ("re-projection grid's X and Y exchanged", "bilinear", _bilinear_xy_exchanged,
     [pins.test_bilinear_reproduces_linear_functions_and_matches_scipy]),
    ("sign of the w-term", "model_vis", _w_sign, [pins.test_wterm_phase_is_the_geometric_delay]),
    ("1/n of Eq. 1 dropped", "model_vis", _w_without_inverse_n, [pins.test_wterm_phase_is_the_geometric_delay]),
    ("Toeplitz kernel conjugated", "psf_kernel", _psf_conjugated, [pins.test_psf_kernel_centre_symmetry_and_normal_matrix]),
    ("feathering weights exchanged", "feather", _feather_weights_exchanged, [pins.test_feather_limits_and_identities]),
    ("Laplacian with a periodic boundary", "laplacian", _laplacian_periodic,
     [pins.test_laplacian_matches_scipy_with_zero_boundary]),
    ("data gradient without the primary beam", "data_cost_grad", _data_gradient_without_beam,
     [pins.test_data_gradient_central_differences]),
    ("Rayleigh-Jeans factor doubled", "rayleigh_jeans_factor", _rj_twice,
     [pins.test_rayleigh_jeans_factor_matches_the_radio_rule_of_thumb]),
]


@pytest.mark.parametrize("what,name,mutate,targets", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_fail_on_a_planted_mistake(monkeypatch, what, name, mutate, targets):
    bad = mutate(getattr(oracle.classic3d, name))
    monkeypatch.setattr(oracle.classic3d, name, bad)
    monkeypatch.setattr(oracle, name, bad)
    for pin in targets:
        with pytest.raises(AssertionError):
            pin()


def test_unet_tap_order_mistake_is_caught(monkeypatch):
    """The network oracle reading the flat vector with dy and dx exchanged."""
    import test_oracle_unet as upins
    from oracle import unet as ou

    def swapped(p, shapes, c):
        out, off = [], 0
        for (ca, _, cb, co, _) in shapes:
            cin = ca + cb
            w = p[off:off + co * 9 * cin].reshape(co, 3, 3, cin).permute(0, 3, 2, 1)
            off += co * 9 * cin
            out.append((w, p[off:off + co]))
            off += co
        return out, p[off:off + c], p[off + c:off + c + 1]

    monkeypatch.setattr(ou, "_unpack_t", swapped)
    with pytest.raises(AssertionError):
        upins.test_flat_layout_tap_order()


def _net_variant(swap_concat=False, avg_pool=False, bilinear_up=False):
    import torch
    import torch.nn.functional as F

    def net(layers, hw, hb, x):
        conv = lambda t, wb: torch.relu(F.conv2d(t, wb[0], wb[1], padding=1))
        if bilinear_up:
            up = lambda t: F.interpolate(t, scale_factor=2, mode="bilinear", align_corners=False)
        else:
            up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
        pool = (lambda t: F.avg_pool2d(t, 2)) if avg_pool else (lambda t: F.max_pool2d(t, 2))
        cat = (lambda deep, skip: torch.cat([skip, deep], 1)) if swap_concat else (lambda deep, skip: torch.cat([deep, skip], 1))
        a0 = conv(x, layers[0]); a1 = conv(a0, layers[1])
        a2 = conv(pool(a1), layers[2]); a3 = conv(a2, layers[3])
        a4 = conv(pool(a3), layers[4]); a5 = conv(a4, layers[5])
        a6 = conv(pool(a5), layers[6]); a7 = conv(a6, layers[7])
        a8 = conv(cat(up(a7), a5), layers[8]); a9 = conv(a8, layers[9])
        a10 = conv(cat(up(a9), a3), layers[10]); a11 = conv(a10, layers[11])
        a12 = conv(cat(up(a11), a1), layers[12]); a13 = conv(a12, layers[13])
        return torch.einsum("bchw,c->bhw", a13, hw) + hb
    return net


NET_MUTANTS = [
    ("skip tensor concatenated first", dict(swap_concat=True), "test_decoder_concatenation_order_by_hand"),
    ("average pooling", dict(avg_pool=True), "test_pooling_is_max_and_upsampling_is_nearest_by_hand"),
    ("bilinear upsampling", dict(bilinear_up=True), "test_pooling_is_max_and_upsampling_is_nearest_by_hand"),
]


@pytest.mark.parametrize("what,kw,pin", NET_MUTANTS, ids=[m[0] for m in NET_MUTANTS])
def test_unet_structure_mistakes_are_caught(monkeypatch, what, kw, pin):
    import test_oracle_unet as upins
    from oracle import unet as ou
    monkeypatch.setattr(ou, "_net", _net_variant(**kw))
    with pytest.raises(AssertionError):
        getattr(upins, pin)()


def test_the_unmutated_network_variant_passes_its_pins(monkeypatch):
    import test_oracle_unet as upins
    from oracle import unet as ou
    monkeypatch.setattr(ou, "_net", _net_variant())
    upins.test_decoder_concatenation_order_by_hand()
    upins.test_pooling_is_max_and_upsampling_is_nearest_by_hand()


def test_solver_without_the_bound_is_caught(monkeypatch):
    """The oracle's L-BFGS-B run without the I >= 0 bound of Eq. 10."""
    orig = oracle.classic3d.solve_lbfgsb

    def unbounded(prob, maxiter, *a, **kw):
        saved = prob.positivity
        prob.positivity = False
        try:
            return orig(prob, maxiter, *a, **kw)
        finally:
            prob.positivity = saved

    monkeypatch.setattr(oracle.classic3d, "solve_lbfgsb", unbounded)
    monkeypatch.setattr(oracle, "solve_lbfgsb", unbounded)
    with pytest.raises(AssertionError):
        pins.test_solver_reaches_nnls_solution_of_tiny_problem()


def test_the_same_pins_pass_on_the_oracle_as_it_is():
    for _, _, _, targets in MUTANTS:
        for pin in targets:
            pin()
