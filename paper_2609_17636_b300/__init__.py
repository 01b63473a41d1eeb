"""B300-native (sm_103a) engine for Classic3D's regularised least-squares cost, its gradient
and its bounded quasi-Newton solve. The compute runs in libivis.so (C ABI: include/ivis.h);
this package only marshals arguments."""
from ._lib import IVIS_FP32, IVIS_FP64, IvisError, load  # noqa: F401
from .engine import Plan, UNet, dirty_image, plan_from_problem, rayleigh_jeans, reproject_grid, unet_planes  # noqa: F401
