"""Thin Python face of the C ABI: one :class:`Plan` per imaging problem.

PyTorch provides device memory and the CUDA stream; the arrays handed over are CUDA
tensors and the calls only pass their pointers and sizes to libivis.so.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import IVIS_FP32, IVIS_FP64, IvisError, SolveReport


def _check(L, plan, status):
    if status != 0:
        msg = L.ivis_last_error(plan)
        raise IvisError(status, msg.decode() if msg else "")


def _dev_f32(t: torch.Tensor, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError("expected a CUDA float32 tensor")
    t = t.contiguous()
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return t


class Plan:
    """One problem: sky cube [nchan, n, n], npoint windows of nb x nb, a data set per
    (pointing, channel) pair, optional single-dish maps. See include/ivis.h."""

    def __init__(self, n: int, nchan: int, npoint: int, nb: int, cell_rad: float,
                 precision: str = "fp32", nufft_tol: float | None = None, kernel_width: int = 0,
                 lambda_r: float = 0.0, lambda_s: float = 0.0, positivity: bool = True,
                 stream: torch.cuda.Stream | None = None, serial_pairs: bool = False,
                 autotune: bool = False, toeplitz: bool = False, wterm: bool = False,
                 grid_tile: int = 0, grid_kernel: int = 0):
        self.L = _lib.load()
        if precision not in ("fp32", "fp64"):
            raise ValueError("precision must be 'fp32' or 'fp64'")
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        if nufft_tol is None:
            nufft_tol = 1e-6 if precision == "fp32" else 1e-11
        self.cfg = _lib.Config(n, nchan, npoint, nb, cell_rad,
                               IVIS_FP32 if precision == "fp32" else IVIS_FP64,
                               nufft_tol, kernel_width, lambda_r, lambda_s, int(bool(positivity)),
                               int(bool(serial_pairs)), int(bool(autotune)), int(bool(toeplitz)),
                               int(bool(wterm)), int(grid_tile), int(grid_kernel))
        self.shape = (nchan, n, n)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._p = ctypes.c_void_p()
        st = self.L.ivis_plan(ctypes.byref(self.cfg), ctypes.c_void_p(self.stream.cuda_stream),
                              ctypes.byref(self._p))
        _check(self.L, None, st)
        self.m = {}

    # ------------------------------------------------------------------ set-up
    def set_pointing(self, k: int, cx: int, cy: int, beam: torch.Tensor):
        beam = _dev_f32(beam, (self.cfg.nb, self.cfg.nb))
        _check(self.L, self._p, self.L.ivis_set_pointing(self._p, k, int(cx), int(cy),
                                                         ctypes.c_void_p(beam.data_ptr())))

    def set_pointing_grid(self, k: int, grid: torch.Tensor | None):
        """Re-project pointing k through sampling locations grid [nb][nb][2] (X, Y)."""
        if grid is None:
            _check(self.L, self._p, self.L.ivis_set_pointing_grid(self._p, k, None))
            return
        grid = _dev_f32(grid, (self.cfg.nb, self.cfg.nb, 2))
        _check(self.L, self._p, self.L.ivis_set_pointing_grid(self._p, k, ctypes.c_void_p(grid.data_ptr())))

    def set_vis(self, k: int, chan: int, uvw: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor):
        m = int(uvw.shape[0])
        if m:
            uvw = _dev_f32(uvw, (m, 3))
            vis = _dev_f32(vis, (m, 2))
            weight = _dev_f32(weight, (m,))
            args = [ctypes.c_void_p(t.data_ptr()) for t in (uvw, vis, weight)]
        else:
            args = [None, None, None]
        _check(self.L, self._p, self.L.ivis_set_vis(self._p, k, chan, m, *args))
        self.m[(k, chan)] = m

    def set_sd(self, chan: int, tsd: torch.Tensor, sigma_sd: float, fwhm_pix: float):
        tsd = _dev_f32(tsd, self.shape[1:])
        _check(self.L, self._p, self.L.ivis_set_sd(self._p, chan, ctypes.c_void_p(tsd.data_ptr()),
                                                   float(sigma_sd), float(fwhm_pix)))

    def prepare(self):
        _check(self.L, self._p, self.L.ivis_prepare(self._p))

    # ------------------------------------------------------------------ evaluation
    def _sky(self, sky: torch.Tensor) -> torch.Tensor:
        if not sky.is_cuda or sky.dtype != self.dtype or tuple(sky.shape) != self.shape:
            raise TypeError(f"sky must be a CUDA {self.dtype} tensor of shape {self.shape}")
        return sky.contiguous()

    def cost_grad(self, sky: torch.Tensor, grad: torch.Tensor | None = None):
        """Returns (Q_tot, gradient tensor, (Q, K, R))."""
        sky = self._sky(sky)
        if grad is None:
            grad = torch.empty_like(sky)
        cost = ctypes.c_double()
        terms = (ctypes.c_double * 3)()
        _check(self.L, self._p, self.L.ivis_cost_grad(self._p, ctypes.c_void_p(sky.data_ptr()),
                                                      ctypes.byref(cost),
                                                      ctypes.c_void_p(grad.data_ptr()), terms))
        return cost.value, grad, (terms[0], terms[1], terms[2])

    def cost_grad_async(self, sky: torch.Tensor, grad: torch.Tensor, cost: torch.Tensor):
        """Enqueue an evaluation on the plan's stream; cost (CUDA float64[4]) receives
        {Q_tot, Q, K, R}. Synchronise with :attr:`cuda_stream` before reading."""
        sky = self._sky(sky)
        _check(self.L, self._p, self.L.ivis_cost_grad_async(
            self._p, ctypes.c_void_p(sky.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
            ctypes.c_void_p(cost.data_ptr())))

    @property
    def cuda_stream(self) -> torch.cuda.ExternalStream:
        ptr = ctypes.c_void_p()
        _check(self.L, self._p, self.L.ivis_get_stream(self._p, ctypes.byref(ptr)))
        return torch.cuda.ExternalStream(ptr.value)

    def cost_grad_host(self, sky_host: torch.Tensor, grad_host: torch.Tensor):
        """Same evaluation from host (ideally pinned) CPU tensors."""
        if sky_host.is_cuda or grad_host.is_cuda:
            raise TypeError("host tensors expected")
        cost = ctypes.c_double()
        terms = (ctypes.c_double * 3)()
        _check(self.L, self._p, self.L.ivis_cost_grad_host(
            self._p, ctypes.c_void_p(sky_host.data_ptr()), ctypes.byref(cost),
            ctypes.c_void_p(grad_host.data_ptr()), terms))
        return cost.value, (terms[0], terms[1], terms[2])

    def predict(self, sky: torch.Tensor, k: int, chan: int) -> torch.Tensor:
        sky = self._sky(sky)
        out = torch.zeros((self.m.get((k, chan), 0), 2), dtype=self.dtype, device=sky.device)
        _check(self.L, self._p, self.L.ivis_predict(self._p, ctypes.c_void_p(sky.data_ptr()), k, chan,
                                                    ctypes.c_void_p(out.data_ptr())))
        return out

    def sd_predict(self, sky: torch.Tensor) -> torch.Tensor:
        sky = self._sky(sky)
        out = torch.empty_like(sky)
        _check(self.L, self._p, self.L.ivis_sd_predict(self._p, ctypes.c_void_p(sky.data_ptr()),
                                                       ctypes.c_void_p(out.data_ptr())))
        return out

    def solve(self, sky: torch.Tensor, maxiter: int, m_hist: int = 10, pgtol: float = 1e-5,
              ftol: float = 1e7 * 2.220446049250313e-16, f_target: float | None = None) -> dict:
        """Overwrites ``sky`` with the solution; returns the solve report. With f_target the
        solve also stops once Q_tot <= f_target."""
        if not sky.is_contiguous():
            raise ValueError("sky must be contiguous (it is updated in place)")
        self._sky(sky)
        rep = SolveReport()
        if f_target is None:
            st = self.L.ivis_solve(self._p, ctypes.c_void_p(sky.data_ptr()), maxiter, m_hist, pgtol,
                                   ftol, ctypes.byref(rep))
        else:
            st = self.L.ivis_solve_target(self._p, ctypes.c_void_p(sky.data_ptr()), maxiter, m_hist,
                                          pgtol, ftol, float(f_target), ctypes.byref(rep))
        _check(self.L, self._p, st)
        return {"iterations": rep.iterations, "evaluations": rep.evaluations, "f": rep.f,
                "pg_inf": rep.pg_inf, "seconds": rep.seconds, "status": rep.status}

    def feather(self, sky: torch.Tensor, sd: torch.Tensor, theta_rad: float,
                sd_scale: float = 1.0) -> torch.Tensor:
        """Short-spacing correction by feathering (ivis_feather): returns a new cube."""
        sky = self._sky(sky)
        sd = _dev_f32(sd, self.shape)
        out = torch.empty_like(sky)
        _check(self.L, self._p, self.L.ivis_feather(self._p, ctypes.c_void_p(sky.data_ptr()),
                                                    ctypes.c_void_p(sd.data_ptr()), float(theta_rad),
                                                    float(sd_scale), ctypes.c_void_p(out.data_ptr())))
        return out

    # ------------------------------------------------------------------ introspection
    def nufft_params(self):
        w, beta, nf = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(self.L, self._p, self.L.ivis_get_nufft_params(self._p, ctypes.byref(w),
                                                             ctypes.byref(beta), ctypes.byref(nf)))
        return w.value, beta.value, nf.value

    def profile(self, enable: bool):
        _check(self.L, self._p, self.L.ivis_profile(self._p, int(bool(enable))))

    def stage_times(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = ctypes.c_int()
        _check(self.L, self._p, self.L.ivis_stage_times(self._p, names, ms, cap, ctypes.byref(cnt)))
        return {names[i].decode(): ms[i] for i in range(min(cnt.value, cap))}

    def tuning(self) -> dict:
        cap, cols = ctypes.c_int(), ctypes.c_int()
        txt = ctypes.c_char_p()
        _check(self.L, self._p, self.L.ivis_tuning(self._p, ctypes.byref(cap), ctypes.byref(cols),
                                                   ctypes.byref(txt)))
        return {"chunk_cap": cap.value, "fft_cols": cols.value,
                "decision": txt.value.decode() if txt.value else ""}

    def launches_per_eval(self) -> int:
        c = ctypes.c_int()
        _check(self.L, self._p, self.L.ivis_launches_per_eval(self._p, ctypes.byref(c)))
        return c.value

    def close(self):
        if self._p:
            self.L.ivis_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_from_problem(prob, precision: str = "fp32", device="cuda", **kw) -> Plan:
    """Build a plan from an object with the attributes of a problem description (n, nchan,
    centres, nb, cell_rad, beams, pairs[k, chan, uvw, vis, weight], lambdas, positivity and,
    for lambda_s != 0, tsd / sigma_sd / sd_fwhm_pix). Host arrays are copied to the device."""
    plan = Plan(prob.n, prob.nchan, prob.centres.shape[0], prob.nb, prob.cell_rad, precision,
                lambda_r=kw.pop("lambda_r", prob.lambda_r), lambda_s=kw.pop("lambda_s", prob.lambda_s),
                positivity=prob.positivity, wterm=kw.pop("wterm", getattr(prob, "wterm", False)), **kw)
    for k in range(prob.centres.shape[0]):
        plan.set_pointing(k, int(prob.centres[k][0]), int(prob.centres[k][1]),
                          torch.as_tensor(prob.beams[k], dtype=torch.float32, device=device))
    for k, g in (getattr(prob, "grids", None) or {}).items():
        plan.set_pointing_grid(k, torch.as_tensor(g, dtype=torch.float32, device=device))
    seen = set()
    for pair in prob.pairs:
        uvw = torch.as_tensor(pair.uvw, dtype=torch.float32, device=device)
        v = torch.view_as_real(torch.as_tensor(pair.vis).to(torch.complex64)).to(device)
        w = torch.as_tensor(pair.weight, dtype=torch.float32, device=device)
        plan.set_vis(pair.k, pair.chan, uvw, v, w)
        seen.add((pair.k, pair.chan))
    for c in range(prob.nchan):
        for k in range(prob.centres.shape[0]):
            if (k, c) not in seen:
                plan.set_vis(k, c, torch.zeros((0, 3), device=device), None, None)
    if plan.cfg.lambda_s != 0.0:
        for c in range(prob.nchan):
            plan.set_sd(c, torch.as_tensor(prob.tsd[c], dtype=torch.float32, device=device),
                        float(prob.sigma_sd[c]), prob.sd_fwhm_pix)
    return plan


class UNet:
    """The learned warm start (ivis_unet_*): [dirty image, beam-weight map] -> initial sky.
    Argument marshalling only; the network runs in libivis.so's kernels."""

    def __init__(self, base_channels: int = 32, max_batch: int = 8, max_hw: int = 256 * 256,
                 stream: torch.cuda.Stream | None = None):
        self.L = _lib.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._p = ctypes.c_void_p()
        st = self.L.ivis_unet_create(base_channels, max_batch, max_hw,
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._p))
        self._check(st, None)
        n = ctypes.c_int64()
        self._check(self.L.ivis_unet_num_params(self._p, ctypes.byref(n)))
        self.nparam = n.value
        self.c = base_channels

    def _check(self, status, plan="self"):
        if status != 0:
            msg = self.L.ivis_unet_last_error(self._p if plan == "self" else None)
            raise IvisError(status, msg.decode() if msg else "")

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.nparam
        self._check(self.L.ivis_unet_set_params(self._p, ctypes.c_void_p(p.ctypes.data)))

    def get_params(self):
        import numpy as np
        p = np.empty(self.nparam, np.float32)
        self._check(self.L.ivis_unet_get_params(self._p, ctypes.c_void_p(p.ctypes.data)))
        return p

    def get_grads(self):
        import numpy as np
        g = np.empty(self.nparam, np.float32)
        self._check(self.L.ivis_unet_get_grads(self._p, ctypes.c_void_p(g.ctypes.data)))
        return g

    def forward(self, inp: torch.Tensor) -> torch.Tensor:
        inp = _dev_f32(inp)
        B, two, H, W = inp.shape
        out = torch.empty((B, H, W), dtype=torch.float32, device=inp.device)
        self._check(self.L.ivis_unet_forward(self._p, ctypes.c_void_p(inp.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), B, H, W))
        return out

    def backward(self, inp: torch.Tensor, tgt: torch.Tensor) -> float:
        inp, tgt = _dev_f32(inp), _dev_f32(tgt)
        B, _, H, W = inp.shape
        loss = ctypes.c_double()
        self._check(self.L.ivis_unet_backward(self._p, ctypes.c_void_p(inp.data_ptr()),
                                              ctypes.c_void_p(tgt.data_ptr()), B, H, W,
                                              ctypes.byref(loss)))
        return loss.value

    def warm_start(self, dirty: torch.Tensor, beamw: torch.Tensor, s0: float, s1: float,
                   s_out: float) -> torch.Tensor:
        """max(s_out * U-Net([s0 dirty, s1 beamw]), 0) for one channel's [H][W] planes, in their
        dtype (ivis_unet_warm_start)."""
        if dirty.dtype != beamw.dtype or dirty.dtype not in (torch.float32, torch.float64):
            raise ValueError("dirty and beam-weight planes must share float32 or float64")
        if dirty.dim() != 2 or beamw.shape != dirty.shape:
            raise ValueError("dirty and beam-weight planes must be [H][W] of one shape")
        if not (dirty.is_cuda and beamw.is_cuda and dirty.is_contiguous() and beamw.is_contiguous()):
            raise ValueError("planes must be contiguous CUDA tensors")
        H, W = dirty.shape
        x0 = torch.empty_like(dirty)
        fp64 = int(dirty.dtype == torch.float64)
        self._check(self.L.ivis_unet_warm_start(self._p, ctypes.c_void_p(dirty.data_ptr()),
                                                ctypes.c_void_p(beamw.data_ptr()), fp64, H, W,
                                                float(s0), float(s1), float(s_out),
                                                ctypes.c_void_p(x0.data_ptr())))
        return x0

    def use_tcgen05(self, enable: bool):
        self._check(self.L.ivis_unet_use_tcgen05(self._p, int(bool(enable))))

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._check(self.L.ivis_unet_adam_step(self._p, lr, beta1, beta2, eps))

    def close(self):
        if self._p:
            self.L.ivis_unet_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unet_planes(a: torch.Tensor, b: torch.Tensor | None, sa: float, sb: float = 1.0) -> torch.Tensor:
    """float32 [2][...] = (sa a, sb b), or [...] = sa a without b (ivis_unet_planes): network
    inputs and targets from the solver's planes."""
    if a.dtype not in (torch.float32, torch.float64) or not (a.is_cuda and a.is_contiguous()):
        raise ValueError("a must be a contiguous float32/float64 CUDA tensor")
    if b is not None and (b.dtype != a.dtype or b.shape != a.shape or not (b.is_cuda and b.is_contiguous())):
        raise ValueError("b must match a in dtype and shape and be contiguous on the device")
    L = _lib.load()
    out = torch.empty(((2,) if b is not None else ()) + tuple(a.shape), dtype=torch.float32, device=a.device)
    st = torch.cuda.current_stream(a.device).cuda_stream
    status = L.ivis_unet_planes(ctypes.c_void_p(a.data_ptr()),
                                ctypes.c_void_p(b.data_ptr() if b is not None else None),
                                int(a.dtype == torch.float64), a.numel(), float(sa), float(sb),
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st))
    if status != 0:
        msg = L.ivis_unet_last_error(None)
        raise IvisError(status, msg.decode() if msg else "")
    return out


def reproject_grid(nb: int, cell_rad: float, ra_k: float, dec_k: float, ra0: float, dec0: float,
                   crpix_x: float, crpix_y: float, sky_proj: str = "SIN"):
    """Re-projection grid float32 [nb][nb][2] (X, Y) of a pointing centred at (ra_k, dec_k)
    (its window a SIN frame) into a sky image of zenithal projection sky_proj ("SIN", "TAN" or
    "ARC") with reference direction (ra0, dec0) at pixel (crpix_x, crpix_y), angles in radians
    (ivis_reproject_grid, computed on the host). Pass it to Plan.set_pointing_grid."""
    import numpy as np
    if sky_proj not in _lib.IVIS_PROJ:
        raise ValueError("sky_proj must be one of " + ", ".join(_lib.IVIS_PROJ))
    L = _lib.load()
    out = np.empty((nb, nb, 2), np.float32)
    status = L.ivis_reproject_grid(int(nb), float(cell_rad), float(ra_k), float(dec_k), float(ra0),
                                   float(dec0), float(crpix_x), float(crpix_y), _lib.IVIS_PROJ[sky_proj],
                                   ctypes.c_void_p(out.ctypes.data))
    if status != 0:
        msg = L.ivis_last_error(None)
        raise IvisError(status, msg.decode() if msg else "")
    return out


def rayleigh_jeans(freq_hz: float) -> float:
    """Jy per square arcsecond per kelvin at freq_hz (ivis_rayleigh_jeans)."""
    return float(_lib.load().ivis_rayleigh_jeans(float(freq_hz)))


def dirty_image(plan: Plan):
    """(-grad Q(0) per channel, beam-weight map) as device tensors (ivis_dirty_image)."""
    d = torch.empty(plan.shape, dtype=plan.dtype, device="cuda")
    b = torch.empty(plan.shape[1:], dtype=plan.dtype, device="cuda")
    _check(plan.L, plan._p, plan.L.ivis_dirty_image(plan._p, ctypes.c_void_p(d.data_ptr()),
                                                    ctypes.c_void_p(b.data_ptr())))
    return d, b
