"""Seeded primitive generators (geometry and random draws only)."""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "C_LIGHT", "HI_FREQ_HZ", "ARCSEC", "DEG", "make_rng", "antenna_layout",
    "baseline_pairs", "uvw_tracks", "gaussian_beam", "point_source_sky",
    "lognormal_sky", "hex_footprint", "flag_keep_mask", "complex_noise",
    "gaussian_noise", "point_source_flux_law", "unet_layer_shapes", "unet_num_params",
    "unet_init", "projection_grid",
]

C_LIGHT = 299_792_458.0
HI_FREQ_HZ = 1.4204058e9
ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def antenna_layout(rng, n_ant: int = 36, diameter_m: float = 6000.0) -> np.ndarray:
    """East/North/Up antenna positions uniform in a disk (metres), shape [n_ant, 3]."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * math.pi * rng.random(n_ant)
    enu = np.zeros((n_ant, 3))
    enu[:, 0] = r * np.cos(th)
    enu[:, 1] = r * np.sin(th)
    return enu


def baseline_pairs(n_ant: int) -> np.ndarray:
    i, j = np.triu_indices(n_ant, k=1)
    return np.stack([i, j], axis=1)


def uvw_tracks(enu: np.ndarray, ha_rad: np.ndarray, dec_rad: float,
               lat_rad: float, freq_hz: float) -> np.ndarray:
    """Earth-rotation uvw in wavelengths for every baseline and hour angle.

    Textbook rotation (Thompson, Moran & Swenson, ch. 4): local ENU baseline
    -> equatorial XYZ at site latitude -> (u, v, w) toward declination
    ``dec`` at hour angle ``H``. Output shape [n_dump * n_baseline, 3],
    dump-major, float64.
    """
    pairs = baseline_pairs(enu.shape[0])
    b = enu[pairs[:, 1]] - enu[pairs[:, 0]]            # [nbl, 3] E, N, U
    e, n, u = b[:, 0], b[:, 1], b[:, 2]
    sl, cl = math.sin(lat_rad), math.cos(lat_rad)
    X = -sl * n + cl * u
    Y = e
    Z = cl * n + sl * u
    lam = C_LIGHT / freq_hz
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    out = []
    for H in np.asarray(ha_rad, dtype=np.float64):
        sh, ch = math.sin(H), math.cos(H)
        uu = sh * X + ch * Y
        vv = -sd * ch * X + sd * sh * Y + cd * Z
        ww = cd * ch * X - cd * sh * Y + sd * Z
        out.append(np.stack([uu, vv, ww], axis=1))
    return np.concatenate(out, axis=0) / lam


def gaussian_beam(nb: int, fwhm_pix: float) -> np.ndarray:
    """Gaussian primary beam on an nb x nb window, peak 1 at pixel (nb/2, nb/2)."""
    s = fwhm_pix / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    c = np.arange(nb) - nb // 2
    g = np.exp(-0.5 * (c / s) ** 2)
    return np.outer(g, g)


def point_source_sky(rng, n: int, nsrc: int, lo: int, hi: int,
                     flux_lo: float, flux_hi: float) -> np.ndarray:
    """nsrc point sources on distinct integer pixels in [lo, hi)^2."""
    sky = np.zeros((n, n))
    cells = rng.choice((hi - lo) * (hi - lo), size=nsrc, replace=False)
    ys, xs = lo + cells // (hi - lo), lo + cells % (hi - lo)
    sky[ys, xs] = rng.uniform(flux_lo, flux_hi, size=nsrc)
    return sky


def lognormal_sky(rng, n: int, slope: float = 3.0, i0: float = 1e-3) -> np.ndarray:
    """Lognormal field exp(g - 1/2) * i0 from a Gaussian field with P(k) ~ k^-slope."""
    white = rng.standard_normal((n, n))
    ky = np.fft.fftfreq(n)[:, None]
    kx = np.fft.fftfreq(n)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (-slope / 2.0)
    g = np.fft.ifft2(np.fft.fft2(white) * amp).real
    g = (g - g.mean()) / g.std()
    return i0 * np.exp(g - 0.5)


def hex_footprint(nrow: int, ncol: int, pitch_pix: float, centre: tuple[float, float]):
    """Close-packed hexagonal pointing centres (odd rows shifted by half a pitch),
    rounded to integer sky pixels; returns int array [nrow*ncol, 2] of (cx, cy)."""
    dy = pitch_pix * math.sqrt(3.0) / 2.0
    pts = []
    for r in range(nrow):
        for c in range(ncol):
            x = (c - (ncol - 1) / 2.0 + (0.5 if r % 2 else 0.0) - 0.25) * pitch_pix
            y = (r - (nrow - 1) / 2.0) * dy
            pts.append((centre[0] + x, centre[1] + y))
    return np.rint(np.array(pts)).astype(np.int64)


def flag_keep_mask(rng, m: int, frac_flagged: float) -> np.ndarray:
    """Boolean keep-mask that removes a uniformly random subset of size round(frac*m)."""
    nflag = int(round(frac_flagged * m))
    keep = np.ones(m, dtype=bool)
    if nflag:
        keep[rng.choice(m, size=nflag, replace=False)] = False
    return keep


def complex_noise(rng, m: int, sigma: float) -> np.ndarray:
    """Complex Gaussian noise, sigma per real and per imaginary component."""
    return sigma * (rng.standard_normal(m) + 1j * rng.standard_normal(m))


def gaussian_noise(rng, shape, sigma: float) -> np.ndarray:
    return sigma * rng.standard_normal(shape)


def point_source_flux_law(freq_hz: np.ndarray, s_ref: float = 5.0,
                          f_ref: float = 1.5e9, alpha: float = -1.0) -> np.ndarray:
    """Power-law input spectrum of the point-source test, S = s_ref (f/f_ref)^alpha."""
    return s_ref * (np.asarray(freq_hz) / f_ref) ** alpha


# ----------------------------------------------------------------- warm-start network shapes
def unet_layer_shapes(c: int = 32):
    """Shapes of the warm-start U-Net's 3x3 layers in parameter order, as tuples
    (cin_a, upsample_a, cin_b, cout, level): encoder 0a, 0b, 1a, 1b, 2a, 2b, 3a, 3b and decoder
    2a, 2b, 1a, 1b, 0a, 0b (decoder 'a' layers read the upsampled deeper tensor, then the skip)."""
    return [(2, 1, 0, c, 0), (c, 1, 0, c, 0),
            (c, 1, 0, 2 * c, 1), (2 * c, 1, 0, 2 * c, 1),
            (2 * c, 1, 0, 4 * c, 2), (4 * c, 1, 0, 4 * c, 2),
            (4 * c, 1, 0, 8 * c, 3), (8 * c, 1, 0, 8 * c, 3),
            (8 * c, 2, 4 * c, 4 * c, 2), (4 * c, 1, 0, 4 * c, 2),
            (4 * c, 2, 2 * c, 2 * c, 1), (2 * c, 1, 0, 2 * c, 1),
            (2 * c, 2, c, c, 0), (c, 1, 0, c, 0)]


def unet_num_params(c: int = 32) -> int:
    n = sum(co * 9 * (ca + cb) + co for (ca, _, cb, co, _) in unet_layer_shapes(c))
    return n + c + 1


def unet_init(c: int = 32, seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, flat float32 vector in the
    library's parameter order."""
    rng = make_rng(seed)
    out = []
    for (ca, _, cb, co, _) in unet_layer_shapes(c):
        fan = 9 * (ca + cb)
        out.append(rng.standard_normal(co * fan) * math.sqrt(2.0 / fan))
        out.append(np.zeros(co))
    out.append(rng.standard_normal(c) * math.sqrt(1.0 / c))
    out.append(np.zeros(1))
    return np.concatenate(out).astype(np.float32)


def projection_grid(nb: int, cx: float, cy: float, rot_rad: float = 0.0, scale: float = 1.0,
                    curvature: float = 0.0) -> np.ndarray:
    """Sampling locations (X, Y) in sky pixels for each window pixel (q, p): a rotation and a
    scale about the pointing centre (cx, cy) (fractional allowed) plus a small quadratic term
    standing in for the SIN projection's departure from the sky grid. float32 [nb][nb][2]."""
    c = np.arange(nb) - nb // 2
    P, Q = np.meshgrid(c, c)
    cr, sr = math.cos(rot_rad), math.sin(rot_rad)
    r2 = (P * P + Q * Q) / float(nb * nb)
    X = cx + scale * (cr * P - sr * Q) * (1.0 + curvature * r2)
    Y = cy + scale * (sr * P + cr * Q) * (1.0 + curvature * r2)
    return np.stack([X, Y], axis=-1).astype(np.float32)
