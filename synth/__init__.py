"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and lays out geometry only: antenna
layouts, Earth-rotation uv tracks, Gaussian primary beams, sky images,
flag masks and noise. It holds none of the method's arithmetic (no Fourier
transform of a sky into visibilities, no convolution by the dish beam, no
cost): the visibilities ``V`` and the single-dish map ``T`` that need the
forward operators are produced by whoever uses these inputs (the oracle in
tests, the library's own predict calls in the benchmark).

Shapes follow the paper's set-ups: a 36-antenna array (ASKAP has 36
antennas, Sect. 5), HI at 1420.4 MHz (Sect. 4.2), Gaussian primary beams of
1 deg FWHM (Sect. 4.3), 6x6 hexagonal footprints (Sect. 4.3), a 16 arcmin
Gaussian single-dish beam (Sect. 4.3) and a point-source law
``S = 5 Jy (nu / 1.5 GHz)^-1`` (Sect. 4.1).
"""
from .generate import *  # noqa: F401,F403
from .workloads import *  # noqa: F401,F403
