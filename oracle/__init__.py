"""FP64 CPU oracle of Classic3D's cost and gradient -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package. It shares no code with the
CUDA path and never imports it.

What it computes (Sect. 2 of the paper, the simplified coplanar forward model):

* window (Eq. 2, the SIN re-projection, which for pointing centres on integer
  sky pixels and a common pixel grid is the identity on the covered pixels):
  ``I'_k[q, p] = I[cy - nb/2 + q, cx - nb/2 + p]`` (zero outside the sky);
* model visibilities (Eq. 3): direct non-uniform DFT of ``A_k * I'_k``
  (``ivis_oracle.c``);
* residual and data term (Eqs. 4-5): ``J_k = 1/2 sum_j w_j |V~_j - V_j|^2``
  with ``w_j = 1/sigma_j^2``; ``Q = sum_k J_k`` (Eq. 6);
* regulariser (Eqs. 7-8): ``R = 1/2 sum_nu ||D I_nu||^2`` with the 5-point
  Laplacian kernel ``d`` and zero boundary;
* fusion term (Eqs. 11-13): ``K = 1/2 sum ((B (x) I) - T)^2 / sigma_sd^2``,
  ``B`` a Gaussian dish beam, truncated at +-ceil(4 sigma_B) pixels and
  normalised to unit sum;
* total (Eq. 14): ``Q_tot = Q + lambda_s K + lambda_r R``;
* analytic gradient of each term (the adjoint operators);
* solver (Eq. 10): scipy's L-BFGS-B, the optimiser the paper calls, with
  bounds ``I >= 0`` when positivity is on and a null initial image.

Beyond the simplified model:

* the general SIN re-projection (Eq. 2) by bilinear interpolation on a
  per-pointing grid of sampling locations, and its adjoint;
* the full visibility equation (Eq. 1): the w-term phase and the 1/n factor
  (``*_w`` functions of ``ivis_oracle.c``, selected by ``prob.wterm``);
* the Toeplitz restatement of the data term (the exact expansion of Eq. 6):
  ``psf_kernel`` and ``toeplitz_data_cost_grad``;
* the appendix's short-spacing feathering and Rayleigh-Jeans factor;
* the learned warm start's network (``oracle/unet.py``; not in the paper).

Pins (``tests/test_oracle_pins.py`` unless named), each against something
other than the oracle itself -- a numpy FFT, scipy, a closed form, brute
force or the paper's printed numbers:

* ``window``, ``window_adjoint``: transpose identity; the bilinear form on an
  integer grid equals the window.
* ``bilinear``, ``bilinear_adjoint``, ``pointing_window*``: scipy
  ``map_coordinates``, exact linear fields, adjoint identity with off-sky and
  non-finite grid entries, central differences of the data gradient.
* ``model_vis``: pure-Python brute force at off-grid uv (nb = 8), a numpy FFT
  on grid-aligned uv, flat phase-centre source,
  phase direction of a one-pixel offset, Hermitian symmetry and 1/cell
  periodicity, linearity; with w: the geometric delay computed in the
  equatorial frame.
* ``adjoint``, ``adjoint_pixels``: pure-Python brute force, adjoint identity to
  1e-13, ``nb^2 ifft2``
  on grid points, pixel subsets equal the full window; with w: adjoint
  identity and central differences.
* ``pair_model_vis``, ``data_cost_grad``, ``data_grad_pixels``: zero cost at
  the noiseless truth, the weighted half square for one visibility, central
  differences, pixel subsets equal the full gradient.
* ``psf_kernel``, ``toeplitz_data_cost_grad``: the explicit normal matrix
  built column by column, equality with the direct data term, the closed form
  of a single zero-spacing visibility.
* ``laplacian``, ``reg_cost_grad``: the paper's kernel (golden file), scipy's
  zero-boundary convolution, the impulse response and hand-derived
  biharmonic stencil (golden file), central differences.
* ``dish_kernel``, ``dish_conv``, ``fusion_cost_grad``: half maximum and
  truncation, scipy ``convolve2d``, flux preservation, zero at a consistent
  map, central differences.
* ``cost_grad``: the weighted sum of the three terms.
* ``solve_lbfgsb``: scipy NNLS on a tiny well-conditioned problem, the
  point-source flux of Sect. 4.1 (one channel, and ten channels against the
  noise-propagated error; a Laplacian spreads it to adjacent pixels), the noise-only behaviour of Sect. 4.2 (noise and
  high spatial frequencies fall as lambda_r grows; noise grows away from the
  pointing centre), the fusion property of
  Sects. 2.4 and 4.3 (the single-dish term restores the large scales and the
  total flux the interferometer misses), and the joint-deconvolution property
  of Sect. 4.3 (a jointly solved mosaic recovers the large scales better than
  a linear mosaic of independently solved pointings).
* ``feather``, ``rayleigh_jeans_factor``: limits and identities of the
  transfer function, an impulse gives the Gaussian, the radio rule of thumb.
* ``unet`` (``tests/test_oracle_unet.py``): parameter count, layers equal
  scipy zero-padded cross-correlation, flat layout, central differences, and a
  hand-built networks whose outputs reveal the decoder's concatenation order,
  max pooling and nearest upsampling.

There is no unpinned function.
"""
from .classic3d import *  # noqa: F401,F403
