"""ivis_sin_grid (host side, no GPU): the re-projection grid of Eq. 2 between two SIN
(orthographic) frames, against the textbook spherical-trigonometry form of the projection
(Calabretta & Greisen 2002) evaluated here independently of the library's rotation matrices."""
import math

import numpy as np
import pytest


def _reference(nb, cell, ra_k, dec_k, ra0, dec0, cx, cy):
    c = (np.arange(nb) - nb // 2) * cell
    l, m = np.meshgrid(c, c)  # l along p (columns), m along q (rows)
    n = np.sqrt(1.0 - l * l - m * m)
    # inverse SIN projection about (ra_k, dec_k): direction (ra, dec)
    dec = np.arcsin(m * math.cos(dec_k) + n * math.sin(dec_k))
    ra = ra_k + np.arctan2(l, n * math.cos(dec_k) - m * math.sin(dec_k))
    # forward SIN projection about (ra0, dec0)
    l1 = np.cos(dec) * np.sin(ra - ra0)
    m1 = np.sin(dec) * math.cos(dec0) - np.cos(dec) * math.sin(dec0) * np.cos(ra - ra0)
    n1 = np.sin(dec) * math.sin(dec0) + np.cos(dec) * math.cos(dec0) * np.cos(ra - ra0)
    X, Y = cx + l1 / cell, cy + m1 / cell
    X[n1 <= 0] = np.nan
    Y[n1 <= 0] = np.nan
    return np.stack([X, Y], axis=-1)


@pytest.mark.parametrize("ra_k,dec_k,ra0,dec0", [
    (1.40, -1.20, 1.40, -1.20),                    # same centre: the integer window
    (1.41, -1.205, 1.40, -1.20),                   # a neighbouring pointing of an LMC mosaic
    (0.02, 0.70, 6.27, 0.69),                      # across RA = 0
    (3.0, 1.45, 3.9, 1.50),                        # near the pole, large RA difference
])
def test_grid_matches_the_spherical_trigonometry_form(ra_k, dec_k, ra0, dec0):
    from paper_2609_17636_b300 import sin_grid
    nb, cell = 64, 7.0 * math.pi / (180 * 3600)
    got = sin_grid(nb, cell, ra_k, dec_k, ra0, dec0, 511.0, 255.5)
    ref = _reference(nb, cell, ra_k, dec_k, ra0, dec0, 511.0, 255.5)
    assert got.dtype == np.float32 and got.shape == (nb, nb, 2)
    assert np.all(np.isfinite(got))
    # float32 storage of pixel coordinates of size up to a few thousand: 1e-3 pixel
    assert np.max(np.abs(got - ref)) <= 1e-3 + 1e-6 * np.max(np.abs(ref)), np.max(np.abs(got - ref))


def test_same_centre_gives_the_integer_window_and_the_centre_maps_to_the_pointing():
    from paper_2609_17636_b300 import sin_grid
    nb, cell = 32, 1e-4
    g = sin_grid(nb, cell, 0.5, 0.3, 0.5, 0.3, 100.0, 60.0)
    P, Q = np.meshgrid(np.arange(nb), np.arange(nb))
    assert np.array_equal(g[..., 0], (100.0 - nb // 2 + P).astype(np.float32))
    assert np.array_equal(g[..., 1], (60.0 - nb // 2 + Q).astype(np.float32))
    # an offset pointing: its window centre lands at its own projected position
    ra_k, dec_k, ra0, dec0 = 0.503, 0.298, 0.5, 0.3
    g = sin_grid(nb, cell, ra_k, dec_k, ra0, dec0, 100.0, 60.0)
    l1 = math.cos(dec_k) * math.sin(ra_k - ra0)
    m1 = math.sin(dec_k) * math.cos(dec0) - math.cos(dec_k) * math.sin(dec0) * math.cos(ra_k - ra0)
    assert abs(g[nb // 2, nb // 2, 0] - (100.0 + l1 / cell)) < 1e-3
    assert abs(g[nb // 2, nb // 2, 1] - (60.0 + m1 / cell)) < 1e-3


def test_far_side_is_nan_and_bad_arguments_are_refused():
    from paper_2609_17636_b300 import IvisError, sin_grid
    g = sin_grid(8, 1e-3, 0.2 + math.pi, -0.4, 0.2, 0.4, 0.0, 0.0)  # the antipode
    assert np.all(np.isnan(g))
    for args in ((0, 1e-3, 0, 0, 0, 0, 0, 0), (8, 0.0, 0, 0, 0, 0, 0, 0), (8, 1e-3, float("nan"), 0, 0, 0, 0, 0)):
        with pytest.raises(IvisError):
            sin_grid(*args)
