"""Placing mosaic pointings on the sky image (the pre-processing of Eq. 2).

A pointing whose SIN frame coincides with the sky grid up to whole pixels is the integer
window of ``ivis_set_pointing`` (exact, deterministic); any other pointing is re-projected
through the grid ``ivis_reproject_grid`` computes. This module chooses between the two and
hands the result to a plan; the grids themselves come from the library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .engine import reproject_grid

__all__ = ["Placement", "place_pointing", "set_pointings"]


@dataclass
class Placement:
    kind: str                 # "window" or "grid"
    cx: int                   # window centre on the sky image (the grid's centre, rounded)
    cy: int
    grid: np.ndarray | None   # float32 [nb][nb][2] for kind == "grid"
    max_offset: float         # largest distance (pixels) between the grid and the integer window


def place_pointing(nb: int, cell_rad: float, ra_k: float, dec_k: float, ra0: float, dec0: float,
                   crpix_x: float, crpix_y: float, sky_proj: str = "SIN", tol_pix: float = 1e-3) -> Placement:
    """Placement of a pointing centred at (ra_k, dec_k) on a sky image of projection sky_proj
    with reference direction (ra0, dec0) at pixel (crpix_x, crpix_y), angles in radians: the
    integer window when every sampling location lies within tol_pix of it, else the grid."""
    grid = reproject_grid(nb, cell_rad, ra_k, dec_k, ra0, dec0, crpix_x, crpix_y, sky_proj)
    centre = grid[nb // 2, nb // 2]
    if not np.all(np.isfinite(centre)):
        raise ValueError("the pointing centre cannot be shown in the sky image's projection")
    cx, cy = (int(np.rint(t)) for t in centre)
    p = np.arange(nb) - nb // 2
    ideal = np.stack(np.meshgrid(cx + p, cy + p), axis=-1).astype(np.float64)
    dev = np.abs(grid.astype(np.float64) - ideal)
    off = float(np.nanmax(dev)) if np.all(np.isfinite(grid)) else float("inf")
    if off <= tol_pix:
        return Placement("window", cx, cy, None, off)
    return Placement("grid", cx, cy, grid, off)


def set_pointings(plan, centres_rad, beams, ra0: float, dec0: float, crpix_x: float, crpix_y: float,
                  sky_proj: str = "SIN", tol_pix: float = 1e-3) -> list:
    """Set every pointing of ``plan`` from its (ra, dec) centre and beam [nb][nb]: the integer
    window where it is exact to tol_pix, the re-projection grid elsewhere. Returns the
    placements."""
    import torch
    nb, cell = plan.cfg.nb, plan.cfg.cell_rad
    out = []
    for k, ((ra_k, dec_k), beam) in enumerate(zip(centres_rad, beams)):
        pl = place_pointing(nb, cell, ra_k, dec_k, ra0, dec0, crpix_x, crpix_y, sky_proj, tol_pix)
        plan.set_pointing(k, pl.cx, pl.cy, torch.as_tensor(np.asarray(beam), dtype=torch.float32, device="cuda"))
        plan.set_pointing_grid(k, None if pl.grid is None else torch.as_tensor(pl.grid, device="cuda"))
        out.append(pl)
    return out
