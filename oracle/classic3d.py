"""Oracle functions (FP64). Test infrastructure only; see the package docstring."""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

__all__ = [
    "lib", "num_threads", "window", "window_adjoint", "model_vis", "adjoint", "adjoint_pixels",
    "pair_model_vis", "data_cost_grad", "data_grad_pixels", "laplacian", "reg_cost_grad",
    "dish_kernel", "dish_conv", "fusion_cost_grad", "cost_grad", "solve_lbfgsb",
    "LAPLACIAN_KERNEL", "bilinear", "bilinear_adjoint", "pointing_window", "pointing_window_adjoint",
    "psf_kernel", "toeplitz_data_cost_grad", "rayleigh_jeans_factor", "feather",
]

# Eq. 7: the Laplacian kernel d of the regulariser.
LAPLACIAN_KERNEL = np.array([[0.0, -1.0, 0.0], [-1.0, 4.0, -1.0], [0.0, -1.0, 0.0]])

_LIB = None


def lib():
    """Load (building first if needed) the oracle's C library."""
    global _LIB
    if _LIB is None:
        from .build import build
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        L.ivo_forward.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int64, dp, dp, dp]
        L.ivo_adjoint.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp, dp, dp]
        L.ivo_adjoint_pixels.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp,
                                         dp, ctypes.c_int64, ip, ip, dp]
        L.ivo_forward_w.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int64, dp, dp, dp, dp]
        L.ivo_adjoint_w.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp, dp, dp, dp]
        L.ivo_adjoint_pixels_w.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp,
                                           dp, dp, ctypes.c_int64, ip, ip, dp]
        L.ivo_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().ivo_num_threads())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- windows (Eq. 2)
def _overlap(c, nb, n):
    """Window index range [a, b) whose sky pixel c - nb/2 + index lies in [0, n)."""
    o = c - nb // 2
    return max(0, -o), min(nb, n - o), o


def window(img: np.ndarray, cx: int, cy: int, nb: int) -> np.ndarray:
    """I'[q, p] = I[cy - nb/2 + q, cx - nb/2 + p], zero where that pixel is off the sky."""
    out = np.zeros((nb, nb))
    qa, qb, oy = _overlap(cy, nb, img.shape[0])
    pa, pb, ox = _overlap(cx, nb, img.shape[1])
    if qa < qb and pa < pb:
        out[qa:qb, pa:pb] = img[oy + qa:oy + qb, ox + pa:ox + pb]
    return out


def window_adjoint(win: np.ndarray, cx: int, cy: int, shape) -> np.ndarray:
    """Transpose of :func:`window`: put the window back on a zero sky of ``shape``."""
    out = np.zeros(shape)
    nb = win.shape[0]
    qa, qb, oy = _overlap(cy, nb, shape[0])
    pa, pb, ox = _overlap(cx, nb, shape[1])
    if qa < qb and pa < pb:
        out[oy + qa:oy + qb, ox + pa:ox + pb] += win[qa:qb, pa:pb]
    return out


def bilinear(img: np.ndarray, grid: np.ndarray) -> np.ndarray:
    """SIN re-projection by bilinear interpolation (Sect. 2.1, Eq. 2; Sect. 3.3): window value
    at (q, p) = the sky interpolated at grid[q, p] = (X, Y) in sky pixel units (X along columns,
    Y along rows), pixels off the sky counting as zero; non-finite grid entries give zero."""
    nb = grid.shape[0]
    out = np.zeros((nb, nb))
    ny, nx = img.shape
    for q in range(nb):
        for p in range(nb):
            X, Y = float(grid[q, p, 0]), float(grid[q, p, 1])
            if not (np.isfinite(X) and np.isfinite(Y)):
                continue
            x0, y0 = int(np.floor(X)), int(np.floor(Y))
            fx, fy = X - x0, Y - y0
            for (dy, dx, wgt) in ((0, 0, (1 - fx) * (1 - fy)), (0, 1, fx * (1 - fy)),
                                  (1, 0, (1 - fx) * fy), (1, 1, fx * fy)):
                y, x = y0 + dy, x0 + dx
                if 0 <= y < ny and 0 <= x < nx:
                    out[q, p] += wgt * img[y, x]
    return out


def bilinear_adjoint(win: np.ndarray, grid: np.ndarray, shape) -> np.ndarray:
    """Transpose of :func:`bilinear`: each window value is spread back with the same weights."""
    out = np.zeros(shape)
    nb = grid.shape[0]
    for q in range(nb):
        for p in range(nb):
            X, Y = float(grid[q, p, 0]), float(grid[q, p, 1])
            if not (np.isfinite(X) and np.isfinite(Y)):
                continue
            x0, y0 = int(np.floor(X)), int(np.floor(Y))
            fx, fy = X - x0, Y - y0
            for (dy, dx, wgt) in ((0, 0, (1 - fx) * (1 - fy)), (0, 1, fx * (1 - fy)),
                                  (1, 0, (1 - fx) * fy), (1, 1, fx * fy)):
                y, x = y0 + dy, x0 + dx
                if 0 <= y < shape[0] and 0 <= x < shape[1]:
                    out[y, x] += wgt * win[q, p]
    return out


def _grid_of(prob, k):
    grids = getattr(prob, "grids", None)
    return None if grids is None else grids.get(k)


def pointing_window(prob, img2d, k):
    """I'_k: the integer window, or the bilinear re-projection when pointing k has a grid."""
    g = _grid_of(prob, k)
    if g is not None:
        return bilinear(img2d, g)
    cx, cy = (int(t) for t in prob.centres[k])
    return window(img2d, cx, cy, prob.nb)


def pointing_window_adjoint(prob, win, k, shape):
    g = _grid_of(prob, k)
    if g is not None:
        return bilinear_adjoint(win, g, shape)
    cx, cy = (int(t) for t in prob.centres[k])
    return window_adjoint(win, cx, cy, shape)


# ------------------------------------------------------------- non-uniform DFT (Eq. 3) and adjoint
def model_vis(f: np.ndarray, cell: float, u: np.ndarray, v: np.ndarray, w=None) -> np.ndarray:
    """Direct DFT  V~_j = sum_{q,p} f[q,p] exp(-2 pi i (u_j l_p + v_j m_q)) (Eq. 3); with w
    given, the full Eq. 1: f / n and the extra phase w_j (n - 1), n = sqrt(1 - l^2 - m^2)."""
    f = _f64(f)
    nb = f.shape[0]
    u, v = _f64(u), _f64(v)
    out = np.zeros(2 * u.shape[0])
    if w is None:
        lib().ivo_forward(nb, cell, _dp(f), u.shape[0], _dp(u), _dp(v), _dp(out))
    else:
        w = _f64(w)
        lib().ivo_forward_w(nb, cell, _dp(f), u.shape[0], _dp(u), _dp(v), _dp(w), _dp(out))
    return out[0::2] + 1j * out[1::2]


def _cvis(c):
    c = np.asarray(c, dtype=np.complex128)
    out = np.empty(2 * c.shape[0])
    out[0::2], out[1::2] = c.real, c.imag
    return out


def adjoint(c: np.ndarray, nb: int, cell: float, u: np.ndarray, v: np.ndarray, w=None) -> np.ndarray:
    """a[q,p] = sum_j c_j exp(+2 pi i (u_j l_p + v_j m_q)) over the whole window; with w given,
    the adjoint of the full Eq. 1 (extra phase +w_j (n - 1), then 1/n)."""
    u, v = _f64(u), _f64(v)
    cv = _cvis(c)
    out = np.zeros(2 * nb * nb)
    if w is None:
        lib().ivo_adjoint(nb, cell, u.shape[0], _dp(u), _dp(v), _dp(cv), _dp(out))
    else:
        w = _f64(w)
        lib().ivo_adjoint_w(nb, cell, u.shape[0], _dp(u), _dp(v), _dp(w), _dp(cv), _dp(out))
    return (out[0::2] + 1j * out[1::2]).reshape(nb, nb)


def adjoint_pixels(c, nb, cell, u, v, qs, ps, w=None) -> np.ndarray:
    u, v = _f64(u), _f64(v)
    cv = _cvis(c)
    qs = np.ascontiguousarray(qs, dtype=np.int32)
    ps = np.ascontiguousarray(ps, dtype=np.int32)
    out = np.zeros(2 * qs.shape[0])
    ip = ctypes.POINTER(ctypes.c_int32)
    if w is None:
        lib().ivo_adjoint_pixels(nb, cell, u.shape[0], _dp(u), _dp(v), _dp(cv), qs.shape[0],
                                 qs.ctypes.data_as(ip), ps.ctypes.data_as(ip), _dp(out))
    else:
        w = _f64(w)
        lib().ivo_adjoint_pixels_w(nb, cell, u.shape[0], _dp(u), _dp(v), _dp(w), _dp(cv), qs.shape[0],
                                   qs.ctypes.data_as(ip), ps.ctypes.data_as(ip), _dp(out))
    return out[0::2] + 1j * out[1::2]


def _wcol(prob, uvw):
    """The w column when the problem uses the full Eq. 1 (prob.wterm), else None."""
    return uvw[:, 2] if getattr(prob, "wterm", False) else None


# -------------------------------------------------------------------- data term (Eqs. 3-6)
def pair_model_vis(prob, sky: np.ndarray, pair, idx=None) -> np.ndarray:
    """Model visibilities of one (pointing, channel) pair for sky cube ``sky``."""
    f = np.asarray(prob.beams[pair.k], dtype=np.float64) * pointing_window(prob, sky[pair.chan], pair.k)
    uvw = pair.uvw if idx is None else pair.uvw[idx]
    return model_vis(f, prob.cell_rad, uvw[:, 0], uvw[:, 1], _wcol(prob, uvw))


def data_cost_grad(prob, sky: np.ndarray, with_grad: bool = True):
    """Q = sum_k J_k (Eqs. 5-6) and its gradient
    dQ/dI = sum_k P_k^T [A_k * Re(sum_j w_j r_j e^{+2 pi i (u l + v m)})]."""
    sky = _f64(sky)
    Q = 0.0
    grad = np.zeros_like(sky) if with_grad else None
    for pair in prob.pairs:
        vt = pair_model_vis(prob, sky, pair)
        r = vt - pair.vis.astype(np.complex128)
        w = pair.weight.astype(np.float64)
        Q += 0.5 * float(np.sum(w * (r.real ** 2 + r.imag ** 2)))
        if with_grad:
            a = adjoint(w * r, prob.nb, prob.cell_rad, pair.uvw[:, 0], pair.uvw[:, 1], _wcol(prob, pair.uvw))
            g = np.asarray(prob.beams[pair.k], dtype=np.float64) * a.real
            grad[pair.chan] += pointing_window_adjoint(prob, g, pair.k, sky.shape[1:])
    return Q, grad


def data_grad_pixels(prob, sky, chan, ys, xs, residuals=None):
    """dQ/dI at the listed sky pixels of channel ``chan`` only (sampled checks). Integer
    windows only: a pointing re-projected through an interpolation grid (Eq. 2) spreads each
    window pixel over four sky pixels, which this sampled form does not follow, so such a
    pointing raises. ``residuals`` (list or dict by pair index) skips recomputing r."""
    sky = _f64(sky)
    out = np.zeros(len(ys))
    for i, pair in enumerate(prob.pairs):
        if pair.chan != chan:
            continue
        if _grid_of(prob, pair.k) is not None:
            raise NotImplementedError("data_grad_pixels: pointing %d uses a re-projection grid" % pair.k)
        cx, cy = (int(t) for t in prob.centres[pair.k])
        q = np.asarray(ys) - (cy - prob.nb // 2)
        p = np.asarray(xs) - (cx - prob.nb // 2)
        inside = (q >= 0) & (q < prob.nb) & (p >= 0) & (p < prob.nb)
        if not inside.any():
            continue
        if residuals is not None:
            r = residuals[i]
        else:
            r = pair_model_vis(prob, sky, pair) - pair.vis.astype(np.complex128)
        w = pair.weight.astype(np.float64)
        a = adjoint_pixels(w * r, prob.nb, prob.cell_rad, pair.uvw[:, 0], pair.uvw[:, 1],
                           q[inside], p[inside], _wcol(prob, pair.uvw))
        out[inside] += np.asarray(prob.beams[pair.k], dtype=np.float64)[q[inside], p[inside]] * a.real
    return out


# ------------------------------------------------- Toeplitz form of the data term (Eqs. 3-6)
def psf_kernel(pair, nb: int, cell: float) -> np.ndarray:
    """T(d) = sum_j w_j exp(+2 pi i (u_j d_x + v_j d_y) cell) for the pixel differences
    d in [-nb, nb)^2, as a [2nb][2nb] array indexed (d_y + nb, d_x + nb): the kernel of the
    normal operator F^H W F of Eqs. 3-5, (F^H W F)[p, q] = T(p - q). It is the adjoint of the
    weights on a 2nb window, whose pixel p' sits at offset p' - nb."""
    w = pair.weight.astype(np.float64)
    return adjoint(w, 2 * nb, cell, pair.uvw[:, 0], pair.uvw[:, 1])


def toeplitz_data_cost_grad(prob, sky: np.ndarray):
    """Q and dQ/dI of Eqs. 5-6 through the expansion, per pair with z = A_k * I'_k,
        Q = 1/2 z.Re(H z) - z.b + 1/2 sum_j w_j |V_j|^2,  dQ/dz = Re(H z) - b,
    H = F^H W F, b = Re(F^H W V). H z is the linear convolution sum_q T(p - q) z[q], taken here
    as a cyclic convolution of period 2nb (numpy FFT) of z, zero-padded to 2nb x 2nb, with T
    wrapped to that period; the entries at d = -nb are never reached and are left out. Equal
    to :func:`data_cost_grad` in exact arithmetic."""
    sky = _f64(sky)
    nb, nf = prob.nb, 2 * prob.nb
    Q = 0.0
    grad = np.zeros_like(sky)
    for pair in prob.pairs:
        A = np.asarray(prob.beams[pair.k], dtype=np.float64)
        z = A * pointing_window(prob, sky[pair.chan], pair.k)
        T = psf_kernel(pair, nb, prob.cell_rad)            # offsets -nb .. nb-1
        T[0, :] = 0.0
        T[:, 0] = 0.0
        Tc = np.roll(T, (-nb, -nb), axis=(0, 1))           # offset d at index d mod nf
        zp = np.zeros((nf, nf))
        zp[:nb, :nb] = z
        Hz = np.fft.ifft2(np.fft.fft2(Tc) * np.fft.fft2(zp))[:nb, :nb]
        w = pair.weight.astype(np.float64)
        V = pair.vis.astype(np.complex128)
        b = adjoint(w * V, nb, prob.cell_rad, pair.uvw[:, 0], pair.uvw[:, 1]).real
        Q += 0.5 * float(np.sum(z * Hz.real)) - float(np.sum(z * b)) + 0.5 * float(np.sum(w * np.abs(V) ** 2))
        grad[pair.chan] += pointing_window_adjoint(prob, A * (Hz.real - b), pair.k, sky.shape[1:])
    return Q, grad


# --------------------------------------------- short-spacing correction by feathering (appendix)
K_BOLTZMANN = 1.380649e-23      # J / K (SI, exact)
C_LIGHT = 299_792_458.0         # m / s (SI, exact)
JANSKY = 1e-26                  # W m^-2 Hz^-1
ARCSEC2_SR = (math.pi / (180.0 * 3600.0)) ** 2


def rayleigh_jeans_factor(freq_hz: float) -> float:
    """Jy arcsec^-2 per kelvin of brightness temperature: I = 2 k nu^2 / c^2 T_B, converted
    from W m^-2 Hz^-1 sr^-1 to Jy per square arcsecond."""
    return 2.0 * K_BOLTZMANN * freq_hz ** 2 / C_LIGHT ** 2 / JANSKY * ARCSEC2_SR


def feather(i_int: np.ndarray, i_sd: np.ndarray, theta_pix: float, sd_scale: float = 1.0):
    """Feathered image of each channel: DFT of both maps on the image grid (no padding),
    I~_comb = B I~_SD + (1 - B) I~_int with the Gaussian transfer function
    B(k) = exp(-2 pi^2 sigma^2 |k|^2), sigma = theta / (2 sqrt(2 ln 2)), k in cycles per pixel
    (theta in pixels), then the inverse DFT (real part). i_sd is multiplied by sd_scale first
    (a unit conversion such as rayleigh_jeans_factor)."""
    i_int = _f64(i_int)
    i_sd = _f64(i_sd) * sd_scale
    n = i_int.shape[-1]
    sig = theta_pix / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    k = np.fft.fftfreq(n)
    B = np.exp(-2.0 * math.pi ** 2 * sig ** 2 * (k[:, None] ** 2 + k[None, :] ** 2))
    out = np.empty_like(i_int)
    for c in range(i_int.shape[0]):
        comb = B * np.fft.fft2(i_sd[c]) + (1.0 - B) * np.fft.fft2(i_int[c])
        out[c] = np.fft.ifft2(comb).real
    return out


# ------------------------------------------------------------------- regulariser (Eqs. 7-8)
def laplacian(img: np.ndarray) -> np.ndarray:
    """D I: convolution with the kernel d (Eq. 7), zero outside the image, same size."""
    img = _f64(img)
    pad = np.zeros((img.shape[0] + 2, img.shape[1] + 2))
    pad[1:-1, 1:-1] = img
    out = np.zeros_like(img)
    for dy in range(3):
        for dx in range(3):
            w = LAPLACIAN_KERNEL[dy, dx]
            if w != 0.0:
                out += w * pad[dy:dy + img.shape[0], dx:dx + img.shape[1]]
    return out


def reg_cost_grad(sky: np.ndarray):
    """R = sum_nu 1/2 ||D I_nu||^2 (Eq. 8); gradient D^T D I_nu (D is symmetric)."""
    R = 0.0
    g = np.zeros_like(_f64(sky))
    for c in range(sky.shape[0]):
        di = laplacian(sky[c])
        R += 0.5 * float(np.sum(di * di))
        g[c] = laplacian(di)
    return R, g


# ------------------------------------------------------------------ fusion term (Eqs. 11-13)
def dish_kernel(fwhm_pix: float) -> np.ndarray:
    """1-D Gaussian dish-beam taps, truncated at +-ceil(4 sigma), unit sum."""
    s = fwhm_pix / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    r = int(math.ceil(4.0 * s))
    t = np.arange(-r, r + 1, dtype=np.float64)
    b = np.exp(-0.5 * (t / s) ** 2)
    return b / b.sum()


def dish_conv(img: np.ndarray, b: np.ndarray) -> np.ndarray:
    """B (x) I with B = b b^T: 'same'-size convolution, zero outside the image."""
    img = _f64(img)
    r = (b.shape[0] - 1) // 2
    ny, nx = img.shape
    pad = np.zeros((ny, nx + 2 * r))
    pad[:, r:r + nx] = img
    rows = np.zeros_like(img)
    for i in range(b.shape[0]):
        rows += b[i] * pad[:, 2 * r - i:2 * r - i + nx]
    pad = np.zeros((ny + 2 * r, nx))
    pad[r:r + ny, :] = rows
    out = np.zeros_like(img)
    for i in range(b.shape[0]):
        out += b[i] * pad[2 * r - i:2 * r - i + ny, :]
    return out


def fusion_cost_grad(sky: np.ndarray, tsd: np.ndarray, sigma_sd, fwhm_pix: float):
    """K = 1/2 sum ((B (x) I - T) / sigma_sd)^2 (Eq. 13); gradient B^T (B (x) I - T)/sigma_sd^2.
    B is symmetric, so B^T is the same convolution."""
    b = dish_kernel(fwhm_pix)
    sig = np.broadcast_to(np.asarray(sigma_sd, dtype=np.float64), (sky.shape[0],))
    K = 0.0
    g = np.zeros_like(_f64(sky))
    for c in range(sky.shape[0]):
        resid = dish_conv(sky[c], b) - tsd[c]
        K += 0.5 * float(np.sum(resid * resid)) / sig[c] ** 2
        g[c] = dish_conv(resid / sig[c] ** 2, b)
    return K, g


# ------------------------------------------------------------------------ total (Eq. 14)
def cost_grad(prob, sky: np.ndarray, tsd=None, sigma_sd=None, with_terms: bool = False):
    """Q_tot = Q + lambda_s K + lambda_r R and its gradient."""
    sky = _f64(sky).reshape(prob.nchan, prob.n, prob.n)
    Q, gQ = data_cost_grad(prob, sky)
    f, g = Q, gQ.copy()
    K = R = 0.0
    if prob.lambda_r != 0.0:
        R, gR = reg_cost_grad(sky)
        f += prob.lambda_r * R
        g += prob.lambda_r * gR
    if prob.lambda_s != 0.0:
        K, gK = fusion_cost_grad(sky, tsd, sigma_sd, prob.sd_fwhm_pix)
        f += prob.lambda_s * K
        g += prob.lambda_s * gK
    if with_terms:
        return f, g, (Q, K, R)
    return f, g


# ---------------------------------------------------------------------- solver (Eq. 10)
def solve_lbfgsb(prob, maxiter: int, m: int = 10, tsd=None, sigma_sd=None, x0=None,
                 pgtol: float = 1e-5, factr: float = 1e7):
    """scipy's L-BFGS-B (the optimiser of Sect. 3.4), null initial image, I >= 0 if
    positivity is on. Returns (x, f, nit, nfev)."""
    from scipy.optimize import minimize
    shape = (prob.nchan, prob.n, prob.n)
    x0 = np.zeros(int(np.prod(shape))) if x0 is None else _f64(x0).ravel()

    def fun(x):
        f, g = cost_grad(prob, x.reshape(shape), tsd, sigma_sd)
        return f, g.ravel()

    bounds = [(0.0, None)] * x0.size if prob.positivity else None
    res = minimize(fun, x0, jac=True, method="L-BFGS-B", bounds=bounds,
                   options={"maxiter": maxiter, "maxcor": m, "gtol": pgtol,
                            "ftol": factr * np.finfo(float).eps})
    return res.x.reshape(shape), float(res.fun), int(res.nit), int(res.nfev)
