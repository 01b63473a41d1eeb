"""Attach the data terms (V, T) to a synthetic problem using the ORACLE's forward operators.

Expected values and inputs of the parity tests never come from the CUDA path: the observed
visibilities are the oracle's direct DFT of the true sky plus the generator's noise draw, and
the single-dish map is the oracle's dish convolution plus noise."""
import numpy as np

import oracle


def attach_data(prob, sky=None, noise=True, sd=True):
    sky = prob.sky_true if sky is None else sky
    for pair in prob.pairs:
        v = oracle.pair_model_vis(prob, sky, pair)
        if noise:
            v = v + pair.noise
        pair.vis = v.astype(np.complex64)
    if sd and prob.sd_fwhm_pix > 0:
        b = oracle.dish_kernel(prob.sd_fwhm_pix)
        t = np.stack([oracle.dish_conv(sky[c], b) for c in range(prob.nchan)])
        sig = prob.sd_noise_frac * np.sqrt(np.mean(t.reshape(prob.nchan, -1) ** 2, axis=1))
        tsd = t + prob.sd_noise_unit * sig[:, None, None]
        prob.tsd = tsd.astype(np.float32)
        prob.sigma_sd = sig
    return prob


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
