"""ivis_reproject_grid (host side, no GPU): the re-projection grid of Eq. 2 from each
pointing's SIN (orthographic) frame into a sky image in a SIN, TAN or ARC projection, against
the textbook spherical-trigonometry forms of those projections (Calabretta & Greisen 2002)
evaluated here independently of the library's rotation matrices."""
import math

import numpy as np
import pytest


def _reference(nb, cell, ra_k, dec_k, ra0, dec0, cx, cy, proj):
    c = (np.arange(nb) - nb // 2) * cell
    l, m = np.meshgrid(c, c)  # l along p (columns), m along q (rows)
    n = np.sqrt(1.0 - l * l - m * m)
    # inverse SIN projection about (ra_k, dec_k): direction (ra, dec)
    dec = np.arcsin(m * math.cos(dec_k) + n * math.sin(dec_k))
    ra = ra_k + np.arctan2(l, n * math.cos(dec_k) - m * math.sin(dec_k))
    # native spherical coordinates about (ra0, dec0): angular distance theta, position angle
    cos_t = np.sin(dec) * math.sin(dec0) + np.cos(dec) * math.cos(dec0) * np.cos(ra - ra0)
    theta = np.arccos(np.clip(cos_t, -1.0, 1.0))
    east = np.cos(dec) * np.sin(ra - ra0)
    north = np.sin(dec) * math.cos(dec0) - np.cos(dec) * math.sin(dec0) * np.cos(ra - ra0)
    pa = np.arctan2(east, north)  # from north through east
    r = {"SIN": np.sin(theta), "TAN": np.tan(theta), "ARC": theta}[proj]
    X, Y = cx + r * np.sin(pa) / cell, cy + r * np.cos(pa) / cell
    bad = cos_t <= 0 if proj in ("SIN", "TAN") else cos_t <= -1 + 1e-12
    X[bad] = np.nan
    Y[bad] = np.nan
    return np.stack([X, Y], axis=-1)


@pytest.mark.parametrize("proj", ["SIN", "TAN", "ARC"])
@pytest.mark.parametrize("ra_k,dec_k,ra0,dec0", [
    (1.40, -1.20, 1.40, -1.20),                    # same centre
    (1.41, -1.205, 1.40, -1.20),                   # a neighbouring pointing of an LMC mosaic
    (0.02, 0.70, 6.27, 0.69),                      # across RA = 0
    (3.0, 1.45, 3.9, 1.50),                        # near the pole, large RA difference
])
def test_grid_matches_the_spherical_trigonometry_form(ra_k, dec_k, ra0, dec0, proj):
    from paper_2609_17636_b300 import reproject_grid
    nb, cell = 64, 7.0 * math.pi / (180 * 3600)
    got = reproject_grid(nb, cell, ra_k, dec_k, ra0, dec0, 511.0, 255.5, proj)
    ref = _reference(nb, cell, ra_k, dec_k, ra0, dec0, 511.0, 255.5, proj)
    assert got.dtype == np.float32 and got.shape == (nb, nb, 2)
    assert np.all(np.isfinite(got))
    # float32 storage of pixel coordinates of size up to a few thousand: 1e-3 pixel
    assert np.max(np.abs(got - ref)) <= 1e-3 + 1e-6 * np.max(np.abs(ref)), np.max(np.abs(got - ref))


def test_same_centre_sin_is_the_integer_window_and_the_centre_maps_to_the_pointing():
    from paper_2609_17636_b300 import reproject_grid
    nb, cell = 32, 1e-4
    g = reproject_grid(nb, cell, 0.5, 0.3, 0.5, 0.3, 100.0, 60.0)
    P, Q = np.meshgrid(np.arange(nb), np.arange(nb))
    assert np.array_equal(g[..., 0], (100.0 - nb // 2 + P).astype(np.float32))
    assert np.array_equal(g[..., 1], (60.0 - nb // 2 + Q).astype(np.float32))
    ra_k, dec_k, ra0, dec0 = 0.503, 0.298, 0.5, 0.3
    g = reproject_grid(nb, cell, ra_k, dec_k, ra0, dec0, 100.0, 60.0)
    l1 = math.cos(dec_k) * math.sin(ra_k - ra0)
    m1 = math.sin(dec_k) * math.cos(dec0) - math.cos(dec_k) * math.sin(dec0) * math.cos(ra_k - ra0)
    assert abs(g[nb // 2, nb // 2, 0] - (100.0 + l1 / cell)) < 1e-3
    assert abs(g[nb // 2, nb // 2, 1] - (60.0 + m1 / cell)) < 1e-3


def test_projections_agree_to_second_order_near_the_reference():
    """SIN, TAN and ARC differ only at third order in the angle from the reference direction."""
    from paper_2609_17636_b300 import reproject_grid
    nb, cell = 16, 1e-6
    g = {p: reproject_grid(nb, cell, 0.1, 0.2, 0.1, 0.2, 0.0, 0.0, p) for p in ("SIN", "TAN", "ARC")}
    assert np.max(np.abs(g["SIN"] - g["TAN"])) < 1e-4 and np.max(np.abs(g["SIN"] - g["ARC"])) < 1e-4


def test_unrepresentable_directions_are_nan_and_bad_arguments_are_refused():
    from paper_2609_17636_b300 import IvisError, reproject_grid
    for proj in ("SIN", "TAN"):  # the antipodal hemisphere
        assert np.all(np.isnan(reproject_grid(8, 1e-3, 0.2 + math.pi, -0.4, 0.2, 0.4, 0.0, 0.0, proj)))
    g = reproject_grid(8, 1e-3, 0.2 + math.pi, -0.3, 0.2, 0.4, 0.0, 0.0, "ARC")  # ARC shows it
    assert np.all(np.isfinite(g))
    for args in ((0, 1e-3, 0, 0, 0, 0, 0, 0), (8, 0.0, 0, 0, 0, 0, 0, 0), (8, 1e-3, float("nan"), 0, 0, 0, 0, 0)):
        with pytest.raises(IvisError):
            reproject_grid(*args)
    with pytest.raises(ValueError):
        reproject_grid(8, 1e-3, 0, 0, 0, 0, 0, 0, "CAR")


def test_pointings_on_the_sky_grid_become_integer_windows_the_others_grids():
    """mosaic.place_pointing: the reference pointing itself is an integer window; a pointing a
    few arcminutes off the reference needs a grid (the SIN frames differ by more than the
    tolerance), and its window centre is its projected position rounded."""
    from paper_2609_17636_b300.mosaic import place_pointing
    nb, cell = 64, 7.0 * math.pi / (180 * 3600)
    same = place_pointing(nb, cell, 1.4, -1.2, 1.4, -1.2, 256.0, 256.0)
    assert same.kind == "window" and (same.cx, same.cy) == (256, 256) and same.max_offset == 0.0
    off = place_pointing(nb, cell, 1.4 + 0.01, -1.2 + 0.003, 1.4, -1.2, 256.0, 256.0)
    assert off.kind == "grid" and off.grid.shape == (nb, nb, 2) and off.max_offset > 1e-3
    c = off.grid[nb // 2, nb // 2]
    assert (off.cx, off.cy) == (int(np.rint(c[0])), int(np.rint(c[1])))
    loose = place_pointing(nb, cell, 1.4 + 0.01, -1.2 + 0.003, 1.4, -1.2, 256.0, 256.0, tol_pix=10.0)
    assert loose.kind == "window" and (loose.cx, loose.cy) == (off.cx, off.cy)
    with pytest.raises(ValueError):  # the antipode cannot be shown
        place_pointing(8, 1e-3, 0.2 + math.pi, -0.4, 0.2, 0.4, 0.0, 0.0)
