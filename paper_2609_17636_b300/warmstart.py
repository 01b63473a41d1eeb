"""Learned warm start: training data from the plain solver, U-Net training, inference.

The network maps [dirty image / sum of weights, beam-weight map] of a channel to that
channel's sky; the solver then starts from max(network output, 0) instead of a null image.
The plain cold-start solve stays the reference: a warm start is judged by the iterations and
wall time it needs to reach the cold start's final cost.

Every step runs in libivis.so (dirty image, input and target scaling, solver, U-Net
forward/backward/Adam, the clamped warm start); this module orchestrates and only moves crops
between tensors.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .engine import Plan, UNet, dirty_image, unet_planes

__all__ = ["SkyProblem", "sky_problem", "TrainingSet", "observe", "make_pairs", "train", "predict_x0",
           "compare_solves"]

I_SCALE = 1e-3  # Jy/pixel: sky values are divided by this inside the network


@dataclass
class SkyProblem:
    """One observation (fixed uv coverage, beams, weights) reused for many skies."""
    plan: Plan
    pairs: list            # [(k, chan, uvw tensor, weight tensor, m)] on the device
    sigma: float           # noise per visibility component
    sum_w: float           # total weight of the channel (normalises the dirty image)


def sky_problem(desc, lambda_r: float, precision: str = "fp32") -> SkyProblem:
    """A single-channel observation from a problem description (n, cell_rad, nb, centres,
    beams, pairs with uvw and weight, sigma_vis); no single-dish term."""
    plan = Plan(desc.n, 1, desc.centres.shape[0], desc.nb, desc.cell_rad, precision,
                lambda_r=lambda_r, lambda_s=0.0, positivity=True)
    for k in range(desc.centres.shape[0]):
        plan.set_pointing(k, int(desc.centres[k][0]), int(desc.centres[k][1]),
                          torch.as_tensor(desc.beams[k], dtype=torch.float32, device="cuda"))
    pairs, sw = [], 0.0
    for pr in desc.pairs:
        if pr.chan != 0:
            continue
        uvw = torch.as_tensor(pr.uvw, dtype=torch.float32, device="cuda")
        w = torch.as_tensor(pr.weight, dtype=torch.float32, device="cuda")
        plan.set_vis(pr.k, 0, uvw, torch.zeros((pr.m, 2), device="cuda"), w)
        pairs.append((pr.k, 0, uvw, w, pr.m))
        sw += float(np.sum(pr.weight, dtype=np.float64))
    return SkyProblem(plan, pairs, float(desc.sigma_vis), sw)


@dataclass
class TrainingSet:
    inputs: list = field(default_factory=list)    # float32 [2][h][w]
    targets: list = field(default_factory=list)   # float32 [h][w]
    solve_seconds: float = 0.0
    solve_iters: list = field(default_factory=list)


def observe(prob: SkyProblem, sky: np.ndarray, rng):
    """Set the plan's visibilities to model(sky) + fresh complex Gaussian noise (same uv
    coverage and weights each time)."""
    p = prob.plan
    xs = torch.as_tensor(sky, dtype=p.dtype, device="cuda").reshape(p.shape)
    for (k, chan, uvw, w, m) in prob.pairs:
        v = p.predict(xs, k, chan).double().cpu().numpy()
        nz = prob.sigma * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
        vis = v[:, 0] + 1j * v[:, 1] + nz
        vt = torch.view_as_real(torch.as_tensor(vis.astype(np.complex64))).cuda()
        p.set_vis(k, chan, uvw, vt, w)


def network_input(prob: SkyProblem):
    """float32 [2][n][n]: dirty image / (sum of weights x I_SCALE), beam-weight map."""
    d, b = dirty_image(prob.plan)
    return unet_planes(d[0], b, 1.0 / (prob.sum_w * I_SCALE), 1.0)


def make_pairs(prob: SkyProblem, skies, crop: int, crops_per_sky: int, maxiter: int, rng,
               ftol: float = 1e-7) -> TrainingSet:
    """For each sky: observe it, solve cold (the target), cut random crops of
    [input planes] -> [solver reconstruction]."""
    ts = TrainingSet()
    p = prob.plan
    n = p.shape[1]
    for sky in skies:
        observe(prob, sky, rng)
        inp = network_input(prob)
        x = torch.zeros(p.shape, dtype=p.dtype, device="cuda")
        t0 = time.perf_counter()
        rep = p.solve(x, maxiter=maxiter, pgtol=0.0, ftol=ftol)
        ts.solve_seconds += time.perf_counter() - t0
        ts.solve_iters.append(rep["iterations"])
        tgt = unet_planes(x[0], None, 1.0 / I_SCALE)
        for _ in range(crops_per_sky):
            y0 = int(rng.integers(0, n - crop + 1))
            x0 = int(rng.integers(0, n - crop + 1))
            ts.inputs.append(inp[:, y0:y0 + crop, x0:x0 + crop].contiguous())
            ts.targets.append(tgt[y0:y0 + crop, x0:x0 + crop].contiguous())
    return ts


def train(net: UNet, ts: TrainingSet, epochs: int, batch: int, lr: float, rng, log=None,
          lr_final: float | None = None):
    """Adam on the MSE loss over shuffled mini-batches; returns the per-epoch mean loss. With
    lr_final, the step size follows a cosine from lr down to lr_final over the whole run."""
    n = len(ts.inputs)
    hist = []
    steps = max(1, epochs * (n // batch))
    step = 0
    for ep in range(epochs):
        order = rng.permutation(n)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = order[b0:b0 + batch]
            xb = torch.stack([ts.inputs[i] for i in idx])
            yb = torch.stack([ts.targets[i] for i in idx])
            tot += net.backward(xb, yb)
            a = lr if lr_final is None else lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * step / steps))
            net.adam_step(a)
            step += 1
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(ep, hist[-1])
    return hist


def predict_x0(net: UNet, prob: SkyProblem) -> torch.Tensor:
    """Initial sky max(I_SCALE U-Net(dirty, beam weight), 0) in the plan's dtype and shape."""
    d, b = dirty_image(prob.plan)
    x0 = net.warm_start(d[0], b, 1.0 / (prob.sum_w * I_SCALE), 1.0, I_SCALE)
    return x0.reshape(prob.plan.shape)


def compare_solves(net: UNet, prob: SkyProblem, sky, rng, maxiter: int, rel_tol: float = 1e-4,
                   ftol: float = 1e-7):
    """Cold solve to convergence, then a warm solve (including inference time) until it reaches
    the cold final cost within rel_tol. Returns a dict of iterations, evaluations, seconds."""
    p = prob.plan
    observe(prob, sky, rng)
    x = torch.zeros(p.shape, dtype=p.dtype, device="cuda")
    cold = p.solve(x, maxiter=maxiter, pgtol=0.0, ftol=ftol)
    target = cold["f"] * (1.0 + rel_tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x0 = predict_x0(net, prob)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    warm = p.solve(x0, maxiter=maxiter, pgtol=0.0, ftol=0.0, f_target=target)
    return {"cold_iters": cold["iterations"], "cold_evals": cold["evaluations"],
            "cold_seconds": cold["seconds"], "cold_f": cold["f"],
            "warm_iters": warm["iterations"], "warm_evals": warm["evaluations"],
            "warm_seconds": warm["seconds"] + t_inf, "warm_f": warm["f"],
            "warm_reached": bool(warm["f"] <= target), "inference_seconds": t_inf}
