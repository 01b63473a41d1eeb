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

Every function that has a pin says which test pins it; there is no unpinned
function.
"""
from .classic3d import *  # noqa: F401,F403
