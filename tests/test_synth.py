"""The seeded input generators follow their stated recipes (CPU).

The synthetic workloads stand in for the paper's CASA and ASKAP data, so what they claim to
be -- array geometry, uv tracks, sky statistics, flagging, noise, footprints -- is checked
here against textbook facts and against the recipe's own numbers."""
import math

import numpy as np

import synth


def test_uvw_tracks_are_a_rotation_of_the_baselines():
    """The (u, v, w) frame is a rotation of the local baseline frame, so every sample keeps
    the baseline's length in wavelengths, whatever the hour angle and declination."""
    rng = synth.make_rng(7)
    enu = synth.antenna_layout(rng, 9, 3000.0)
    enu[:, 2] = rng.uniform(-20.0, 20.0, 9)  # some height differences too
    ha = np.linspace(-4.0, 4.0, 11) * 15.0 * synth.DEG
    lam = synth.C_LIGHT / synth.HI_FREQ_HZ
    for dec, lat in ((synth.DEC_LMC_RAD, synth.LAT_ASKAP_RAD), (40.7 * synth.DEG, 34.1 * synth.DEG)):
        uvw = synth.uvw_tracks(enu, ha, dec, lat, synth.HI_FREQ_HZ)
        pairs = synth.baseline_pairs(9)
        blen = np.linalg.norm(enu[pairs[:, 1]] - enu[pairs[:, 0]], axis=1) / lam
        assert uvw.shape == (len(ha) * len(pairs), 3)
        assert np.allclose(np.linalg.norm(uvw, axis=1), np.tile(blen, len(ha)), rtol=1e-12)


def test_east_west_baseline_traces_the_textbook_ellipse():
    """An east-west baseline of length b draws u = b cos H, v = b sin(dec) sin H (in
    wavelengths), an ellipse of axis ratio sin(dec), with u = b, v = w = 0 at transit."""
    b = 750.0
    enu = np.array([[0.0, 0.0, 0.0], [b, 0.0, 0.0]])
    ha = np.linspace(-6.0, 6.0, 25) * 15.0 * synth.DEG
    dec = -69.0 * synth.DEG
    uvw = synth.uvw_tracks(enu, ha, dec, synth.LAT_ASKAP_RAD, synth.HI_FREQ_HZ)
    bl = b * synth.HI_FREQ_HZ / synth.C_LIGHT
    assert np.allclose(uvw[:, 0], bl * np.cos(ha), atol=1e-9 * bl)
    assert np.allclose(uvw[:, 1], bl * math.sin(dec) * np.sin(ha), atol=1e-9 * bl)
    mid = len(ha) // 2
    assert abs(uvw[mid, 0] - bl) < 1e-9 * bl and abs(uvw[mid, 1]) < 1e-9 * bl and abs(uvw[mid, 2]) < 1e-9 * bl


def test_lognormal_sky_has_the_stated_statistics():
    """I = i0 exp(g - 1/2) with g a zero-mean, unit-variance Gaussian field of power spectrum
    k^-3: log(I / i0) + 1/2 has mean 0 and variance 1 exactly, and its azimuthally averaged
    power falls with a log-log slope near -3."""
    n = 256
    sky = synth.lognormal_sky(synth.make_rng(3), n, slope=3.0, i0=1e-3)
    g = np.log(sky / 1e-3) + 0.5
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    P = np.abs(np.fft.fft2(g)) ** 2
    k = np.hypot(np.fft.fftfreq(n)[:, None], np.fft.fftfreq(n)[None, :]) * n
    ks = np.arange(4, 64)
    pk = np.array([P[(k >= a) & (k < a + 1)].mean() for a in ks])
    slope = np.polyfit(np.log(ks + 0.5), np.log(pk), 1)[0]
    assert abs(slope + 3.0) < 0.3, slope


def test_gaussian_beam_half_maximum_and_peak():
    beam = synth.gaussian_beam(64, 10.0)
    assert beam[32, 32] == 1.0
    assert abs(beam[32, 37] - 0.5) < 1e-12 and abs(beam[27, 32] - 0.5) < 1e-12


def test_flagging_removes_exactly_the_stated_fraction():
    keep = synth.flag_keep_mask(synth.make_rng(4), 10_000, 0.23)
    assert keep.sum() == 7700


def test_config_c1_recipe():
    prob = synth.config_c1()
    assert (prob.n, prob.nb, prob.nchan, prob.npoint) == (128, 128, 1, 1)
    assert prob.total_vis == 630 * 13 == 8190
    ys, xs = np.nonzero(prob.sky_true[0])
    assert len(ys) == 5 and ys.min() >= 16 and ys.max() < 112 and xs.min() >= 16 and xs.max() < 112
    f = prob.sky_true[0][ys, xs]
    assert f.min() >= 0.1 and f.max() <= 1.0
    pair = prob.pairs[0]
    assert np.all(pair.weight == np.float32(1e6))
    assert abs(np.std(pair.noise.real) - 1e-3) < 0.05e-3 and abs(np.std(pair.noise.imag) - 1e-3) < 0.05e-3
    assert abs(prob.cell_rad / synth.ARCSEC - 4.0) < 1e-12 and (prob.lambda_r, prob.lambda_s) == (0.0, 0.0)


def test_config_c2_recipe():
    prob = synth.config_c2()
    cell = prob.cell_rad
    assert (prob.n, prob.nb, prob.npoint, prob.nchan) == (512, 512, 7, 1)
    assert abs(cell / synth.ARCSEC - 7.0) < 1e-12
    # hexagonal footprint: a centre and six neighbours at the 0.3 deg pitch, 60 deg apart
    c = prob.centres.astype(np.float64)
    d = c[1:] - c[0]
    pitch = 0.3 * synth.DEG / cell
    assert np.all(np.abs(np.hypot(d[:, 0], d[:, 1]) - pitch) <= 0.75)
    ang = np.sort(np.degrees(np.arctan2(d[:, 1], d[:, 0])) % 360.0)
    assert np.all(np.abs(np.diff(ang) - 60.0) < 0.5)
    # 630 baselines x 360 dumps per pointing, 0-30 % of them flagged
    for pair in prob.pairs:
        kept = pair.m / (630 * 360)
        assert 0.7 - 1e-9 <= kept <= 1.0
    assert 0.7 * 7 * 226_800 < prob.total_vis < 7 * 226_800
    # beams of 0.3 deg FWHM, the 16 arcmin dish, the lognormal sky at 1 mJy per pixel
    fwhm_pix = 0.3 * synth.DEG / cell
    b = prob.beams[0].astype(np.float64)
    prof = b[256, 256:]
    half = np.interp(0.5, prof[::-1], np.arange(256)[::-1])
    assert abs(2 * half - fwhm_pix) < 0.5
    assert abs(prob.sd_fwhm_pix - 16.0 * 60.0 / 7.0) < 1e-9
    assert prob.sky_true.min() > 0 and abs(prob.sky_true.mean() / 1e-3 - 1.0) < 0.25
    assert prob.lambda_s == 1.0 and prob.positivity


def test_point_source_spectrum_workload_recipe():
    prob = synth.point_source_spectrum()
    assert prob.nchan == 10 and np.allclose(prob.freqs_hz, 0.55e9 + 0.1e9 * np.arange(10))
    assert np.allclose(prob.sky_true[:, 8, 8], 5.0 * (prob.freqs_hz / 1.5e9) ** -1.0)
    assert all(p.m == 351 * 18 and p.chan == c for c, p in enumerate(prob.pairs))
    # uv scale with frequency: the same baselines at each channel
    r = np.linalg.norm(prob.pairs[9].uvw.astype(np.float64), axis=1) / np.linalg.norm(
        prob.pairs[0].uvw.astype(np.float64), axis=1)
    assert np.allclose(r, 1.45 / 0.55, rtol=1e-6)
