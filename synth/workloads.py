"""Workload descriptions: the inputs of one imaging problem, without its data term.

A :class:`Problem` carries everything a user hands to the imager except the
observed visibilities ``V`` and the single-dish map ``T`` (those need the
forward operators; see the package docstring). ``noise`` holds the complex
noise draw for each (pointing, channel) pair and ``sd_noise_unit`` a unit
normal draw for the single-dish map; the caller scales and adds them.

Every array that crosses into the library is already rounded to the
precision the library's boundary takes (float32 uvw, weights and
visibilities), so the oracle and the GPU path see bit-identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .generate import (ARCSEC, DEG, HI_FREQ_HZ, antenna_layout, complex_noise,
                       flag_keep_mask, gaussian_beam, hex_footprint, lognormal_sky,
                       make_rng, point_source_flux_law, point_source_sky, uvw_tracks)

__all__ = ["VisSet", "Problem", "config_c1", "config_c2", "config_c3", "config_c4",
           "small_mosaic", "point_source_spectrum", "LAT_ASKAP_RAD", "DEC_LMC_RAD",
           "SPECTRUM_FREQS_HZ"]

LAT_ASKAP_RAD = -26.7 * DEG
DEC_LMC_RAD = -69.0 * DEG
# channel centres of the multi-frequency point-source observation (Sect. 4.1): one window
# centred at 1.0 GHz, 1.0 GHz wide, ten equal channels
SPECTRUM_FREQS_HZ = 0.55e9 + 0.1e9 * np.arange(10)


@dataclass
class VisSet:
    """Visibilities of one (pointing k, channel) pair, in caller order."""
    k: int
    chan: int
    uvw: np.ndarray        # float32 [m, 3], wavelengths
    weight: np.ndarray     # float32 [m], natural weights 1/sigma^2
    noise: np.ndarray      # complex128 [m], complex noise draw (sigma per component)
    vis: np.ndarray | None = None   # complex64 [m]: filled by the caller

    @property
    def m(self) -> int:
        return int(self.uvw.shape[0])


@dataclass
class Problem:
    name: str
    n: int                       # sky is n x n per channel
    cell_rad: float
    nchan: int
    nb: int                      # pointing window nb x nb (power of two)
    centres: np.ndarray          # int64 [npoint, 2]: (cx, cy) sky pixel of each window centre
    beams: np.ndarray            # float32 [npoint, nb, nb]
    pairs: list                  # list[VisSet]
    sky_true: np.ndarray         # float64 [nchan, n, n]
    lambda_r: float = 0.0
    lambda_s: float = 0.0
    positivity: bool = True
    sd_fwhm_pix: float = 0.0     # single-dish beam FWHM in pixels (0: no fusion term)
    sd_noise_frac: float = 0.05
    sd_noise_unit: np.ndarray | None = None   # float64 [nchan, n, n], unit normal draw
    sigma_vis: float = 1e-3
    freqs_hz: np.ndarray = field(default_factory=lambda: np.array([HI_FREQ_HZ]))
    wterm: bool = False          # model the full Eq. 1 (w-term and 1/n) instead of Eq. 3

    @property
    def npoint(self) -> int:
        return int(self.centres.shape[0])

    @property
    def total_vis(self) -> int:
        return int(sum(p.m for p in self.pairs))


def _as_f32_uvw(uvw: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(uvw, dtype=np.float32)


def _vis_set(rng, k, chan, uvw64, sigma, keep=None):
    if keep is not None:
        uvw64 = uvw64[keep]
    m = uvw64.shape[0]
    w = np.full(m, 1.0 / (sigma * sigma), dtype=np.float32)
    return VisSet(k=k, chan=chan, uvw=_as_f32_uvw(uvw64), weight=w,
                  noise=complex_noise(rng, m, sigma))


def config_c1(seed: int = 1001) -> Problem:
    """Plain single pointing: 128^2 sky at 4 arcsec, one 1 deg Gaussian beam,
    36 antennas in 6 km -> 630 baselines x 13 dumps over +-5 h = 8190 visibilities,
    5 point sources U[0.1, 1] Jy, noise 1 mJy, no regularisation, positivity."""
    rng = make_rng(seed)
    n, nb = 128, 128
    cell = 4.0 * ARCSEC
    enu = antenna_layout(rng, 36, 6000.0)
    ha = np.linspace(-5.0, 5.0, 13) * (15.0 * DEG)
    uvw = uvw_tracks(enu, ha, DEC_LMC_RAD, LAT_ASKAP_RAD, HI_FREQ_HZ)
    sky = point_source_sky(rng, n, 5, 16, 112, 0.1, 1.0)[None]
    beam = gaussian_beam(nb, 1.0 * DEG / cell).astype(np.float32)[None]
    pairs = [_vis_set(rng, 0, 0, uvw, 1e-3)]
    return Problem("c1_single_pointing", n, cell, 1, nb, np.array([[n // 2, n // 2]]),
                   beam, pairs, sky, lambda_r=0.0, lambda_s=0.0, positivity=True,
                   sigma_vis=1e-3)


def point_source_spectrum(seed: int = 1010, n: int = 16, cell_arcsec: float = 120.0,
                          sigma: float = 0.1) -> Problem:
    """Stand-in for the multi-frequency point-source observation of Sect. 4.1: one pointing,
    27 antennas in a 1 km disk (a compact, VLA-D-sized array), +-5 h around transit in 2000 s
    integrations (18 dumps) at declination +40.7 deg from latitude +34.1 deg, ten channels
    (SPECTRUM_FREQS_HZ), a point source at the phase centre with S = 5 Jy (nu / 1.5 GHz)^-1,
    Gaussian noise sigma per real and imaginary component, natural weights, a 45' Gaussian
    beam, no regularisation, positivity. The pixel (2' by default) is coarser than the
    synthesised beam at every channel, so the source is unresolved in the pixel basis."""
    rng = make_rng(seed)
    cell = cell_arcsec * ARCSEC
    enu = antenna_layout(rng, 27, 1000.0)
    ha = (np.arange(18) + 0.5 - 9.0) * (2000.0 / 86400.0) * (2.0 * math.pi)
    dec, lat = 40.73 * DEG, 34.08 * DEG
    flux = point_source_flux_law(SPECTRUM_FREQS_HZ)
    sky = np.zeros((SPECTRUM_FREQS_HZ.size, n, n))
    sky[:, n // 2, n // 2] = flux
    pairs = [_vis_set(rng, 0, c, uvw_tracks(enu, ha, dec, lat, f), sigma)
             for c, f in enumerate(SPECTRUM_FREQS_HZ)]
    beam = gaussian_beam(n, 45.0 * 60.0 * ARCSEC / cell).astype(np.float32)[None]
    return Problem("point_source_spectrum", n, cell, SPECTRUM_FREQS_HZ.size, n,
                   np.array([[n // 2, n // 2]]), beam, pairs, sky, lambda_r=0.0, lambda_s=0.0,
                   positivity=True, sigma_vis=sigma, freqs_hz=SPECTRUM_FREQS_HZ.copy())


def config_c2(seed: int = 1002, lambda_r: float = 1e-2, dumps: int = 360) -> Problem:
    """7-pointing hexagonal mosaic: 512^2 sky at 7 arcsec, 0.3 deg beams at 0.3 deg
    pitch, 630 baselines x 360 dumps (1 h, 10 s) per pointing, 0-30 % flagging,
    lognormal k^-3 sky, Laplacian lambda_r, fusion with a 16 arcmin dish (lambda_s = 1)."""
    rng = make_rng(seed)
    n, nb = 512, 512
    cell = 7.0 * ARCSEC
    fwhm = 0.3 * DEG / cell
    pitch = 0.3 * DEG / cell
    c = n // 2
    centres = [(c, c)]
    for a in range(6):
        th = a * math.pi / 3.0
        centres.append((c + pitch * math.cos(th), c + pitch * math.sin(th)))
    centres = np.rint(np.array(centres)).astype(np.int64)
    enu = antenna_layout(rng, 36, 6000.0)
    ha = np.linspace(-0.5, 0.5, dumps) * (15.0 * DEG)
    uvw = uvw_tracks(enu, ha, DEC_LMC_RAD, LAT_ASKAP_RAD, HI_FREQ_HZ)
    beam1 = gaussian_beam(nb, fwhm).astype(np.float32)
    beams = np.repeat(beam1[None], len(centres), axis=0)
    sky = lognormal_sky(rng, n)[None]
    pairs = []
    for k in range(len(centres)):
        keep = flag_keep_mask(rng, uvw.shape[0], rng.uniform(0.0, 0.3))
        pairs.append(_vis_set(rng, k, 0, uvw, 1e-3, keep))
    return Problem("c2_hex7_mosaic", n, cell, 1, nb, centres, beams, pairs, sky,
                   lambda_r=lambda_r, lambda_s=1.0, positivity=True,
                   sd_fwhm_pix=16.0 * 60.0 * ARCSEC / cell,
                   sd_noise_unit=rng.standard_normal((1, n, n)), sigma_vis=1e-3)


def config_c3(seed: int = 1003, nchan: int = 32, nrow: int = 6, ncol: int = 6) -> Problem:
    """Batched cube: 1024^2 sky at 25 arcsec, 36 beams on a 6x6 hexagonal footprint
    (0.9 deg pitch, 1 deg FWHM), nb = 512, 32 channels spaced 18.5 kHz, uneven
    U[1e5, 3e5] visibilities per (beam, channel) drawn from 630 x 476 dumps,
    lognormal k^-3 sky with Gaussian line profiles."""
    rng = make_rng(seed)
    n, nb = 1024, 512
    cell = 25.0 * ARCSEC
    centres = hex_footprint(nrow, ncol, 0.9 * DEG / cell, (n / 2, n / 2))
    beam1 = gaussian_beam(nb, 1.0 * DEG / cell).astype(np.float32)
    beams = np.repeat(beam1[None], centres.shape[0], axis=0)
    enu = antenna_layout(rng, 36, 6000.0)
    ha = np.linspace(-5.0, 5.0, 476) * (15.0 * DEG)
    uvw0 = uvw_tracks(enu, ha, DEC_LMC_RAD, LAT_ASKAP_RAD, HI_FREQ_HZ)
    freqs = HI_FREQ_HZ + 18.5e3 * np.arange(nchan)
    L = lognormal_sky(rng, n)
    c0 = lognormal_sky(rng, n)
    c0 = 8.0 + 16.0 * (c0 - c0.min()) / (c0.max() - c0.min())
    ch = np.arange(nchan)[:, None, None]
    sky = L[None] * np.exp(-((ch - c0[None]) ** 2) / (2.0 * 4.0 ** 2))
    pairs = []
    mtot = uvw0.shape[0]
    for chn in range(nchan):
        scale = freqs[chn] / HI_FREQ_HZ
        for k in range(centres.shape[0]):
            m = int(rng.integers(100_000, 300_001))
            sel = np.sort(rng.choice(mtot, size=m, replace=False))
            pairs.append(_vis_set(rng, k, chn, uvw0[sel] * scale, 1e-3))
    return Problem("c3_batched_cube", n, cell, nchan, nb, centres, beams, pairs, sky,
                   lambda_r=1e-2, lambda_s=0.0, positivity=True, sigma_vis=1e-3,
                   freqs_hz=freqs)


def config_c4(seed: int = 1004, dumps: int = 3600) -> Problem:
    """Full footprint, 10 h: 4096^2 sky at 5 arcsec, 36 beams (6x6 hex, 0.9 deg pitch,
    1 deg FWHM), nb = 2048, 630 baselines x 3600 dumps = 2.27e6 visibilities per beam,
    lambda_r = 1e-2 plus fusion with a 16 arcmin dish."""
    rng = make_rng(seed)
    n, nb = 4096, 2048
    cell = 5.0 * ARCSEC
    centres = hex_footprint(6, 6, 0.9 * DEG / cell, (n / 2, n / 2))
    beam1 = gaussian_beam(nb, 1.0 * DEG / cell).astype(np.float32)
    beams = np.repeat(beam1[None], centres.shape[0], axis=0)
    enu = antenna_layout(rng, 36, 6000.0)
    ha = np.linspace(-5.0, 5.0, dumps) * (15.0 * DEG)
    uvw = uvw_tracks(enu, ha, DEC_LMC_RAD, LAT_ASKAP_RAD, HI_FREQ_HZ)
    sky = lognormal_sky(rng, n)[None]
    pairs = [_vis_set(rng, k, 0, uvw, 1e-3) for k in range(centres.shape[0])]
    return Problem("c4_full_footprint", n, cell, 1, nb, centres, beams, pairs, sky,
                   lambda_r=1e-2, lambda_s=1.0, positivity=True,
                   sd_fwhm_pix=16.0 * 60.0 * ARCSEC / cell,
                   sd_noise_unit=rng.standard_normal((1, n, n)), sigma_vis=1e-3)


def small_mosaic(seed: int, n: int = 96, nb: int = 64, nchan: int = 2, npoint: int = 3,
                 ndump: int = 6, n_ant: int = 12, cell_arcsec: float = 20.0,
                 lambda_r: float = 0.1, lambda_s: float = 0.5, sd_fwhm_pix: float = 6.0,
                 ragged: bool = True, sky_kind: str = "lognormal") -> Problem:
    """Small multi-pointing, multi-channel problem the oracle finishes in seconds.

    Windows extend past the sky edge (zero padding is exercised), counts are
    ragged per pair, baselines exceed the pixel Nyquist limit (folding)."""
    rng = make_rng(seed)
    cell = cell_arcsec * ARCSEC
    enu = antenna_layout(rng, n_ant, 6000.0)
    ha = np.linspace(-4.0, 4.0, ndump) * (15.0 * DEG)
    uvw0 = uvw_tracks(enu, ha, DEC_LMC_RAD, LAT_ASKAP_RAD, HI_FREQ_HZ)
    centres = np.stack([rng.integers(nb // 4, n - nb // 4, npoint),
                        rng.integers(nb // 4, n - nb // 4, npoint)], axis=1).astype(np.int64)
    fw = 0.6 * nb
    beams = np.stack([gaussian_beam(nb, fw * (1.0 + 0.1 * k)) for k in range(npoint)]
                     ).astype(np.float32)
    if sky_kind == "lognormal":
        sky = np.stack([lognormal_sky(rng, n, i0=1.0) for _ in range(nchan)])
    else:
        sky = np.stack([point_source_sky(rng, n, 4, 8, n - 8, 0.1, 1.0) for _ in range(nchan)])
    pairs = []
    for chn in range(nchan):
        for k in range(npoint):
            keep = flag_keep_mask(rng, uvw0.shape[0], rng.uniform(0.0, 0.4) if ragged else 0.0)
            vs = _vis_set(rng, k, chn, uvw0 * (1.0 + 0.01 * chn), 0.05, keep)
            vs.weight = (vs.weight * rng.uniform(0.5, 1.5, vs.m)).astype(np.float32)
            pairs.append(vs)
    return Problem(f"small_mosaic_{seed}", n, cell, nchan, nb, centres, beams, pairs, sky,
                   lambda_r=lambda_r, lambda_s=lambda_s, positivity=True,
                   sd_fwhm_pix=sd_fwhm_pix,
                   sd_noise_unit=rng.standard_normal((nchan, n, n)), sigma_vis=0.05)
