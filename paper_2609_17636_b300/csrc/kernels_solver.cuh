// kernels_solver.cuh -- device side of the bounded limited-memory quasi-Newton solve (a10).
//
// The paper minimises Q_tot with L-BFGS-B (Eq. 10; Zhu et al. 1997) under I >= 0. Here the
// inverse-Hessian approximation is applied in the compact form of Byrd, Nocedal & Schnabel
// (1994): H = gamma I + [S  gamma Y] M [S^T; gamma Y^T], so one direction needs the 2m inner
// products S^T g_F, Y^T g_F (one pass over the history) and one combination pass. The free
// set F = {i : not (I_i <= 0 and g_i > 0)} restricts the step to variables that can move
// (projected quasi-Newton); the step is projected onto I >= 0 and accepted by an Armijo test
// on the projected path. Every inner product (the 2m + 1 of the direction, g.d, the Armijo
// slope and the 3m of a new pair) is accumulated in FP64 from its first term: each product of
// two working-precision values is formed exactly in FP64 (24 + 24 bits fit its 53) and summed
// in FP64 within the thread, the warp and the CTA. History vectors and the per-pixel
// arithmetic of d and of the trial point stay in the plan's real type.
#pragma once
#include "common.cuh"

namespace ivis {

constexpr int SOL_MAXM = 32;
constexpr int SOL_CHUNK = 1024;  // pixels per CTA in the solver passes

struct SlotList {
    int m;
    int slot[SOL_MAXM];
};

struct SolverBufs {
    int mcap = 0;
    size_t npix = 0;
    int nblk = 0;
    void *S = nullptr, *Y = nullptr, *xk = nullptr, *gk = nullptr, *d = nullptr;
    double *SY = nullptr, *YY = nullptr;  // [mcap][mcap] by slot
    double *part = nullptr;               // [nblk][3 * mcap + 4]
    double *coef = nullptr;               // [2 * mcap]
    double *scal = nullptr;               // see k_sol_* below
    double *scal_h = nullptr;             // pinned mirror of scal
};

inline void solver_free(SolverBufs &b) {
    void *ptrs[] = {b.S, b.Y, b.xk, b.gk, b.d, b.SY, b.YY, b.part, b.coef, b.scal};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (b.scal_h) cudaFreeHost(b.scal_h);
    b = SolverBufs{};
}

// Allocation of the per-problem solver buffers happens on first use (ivis_solve).
template <typename T>
inline ivis_status solver_alloc(SolverBufs &b, size_t npix) {
    solver_free(b);
    b.npix = npix;
    b.nblk = (int)((npix + SOL_CHUNK - 1) / SOL_CHUNK);
    return IVIS_OK;
}

template <typename T>
inline ivis_status solver_ensure(SolverBufs &b, int m) {
    if (b.mcap >= m && b.S) return IVIS_OK;
    size_t npix = b.npix;
    int nblk = b.nblk;
    solver_free(b);
    b.npix = npix;
    b.nblk = nblk;
    b.mcap = m;
    size_t v = npix * sizeof(T);
    bool ok = cudaMalloc(&b.S, v * m) == cudaSuccess && cudaMalloc(&b.Y, v * m) == cudaSuccess &&
              cudaMalloc(&b.xk, v) == cudaSuccess && cudaMalloc(&b.gk, v) == cudaSuccess &&
              cudaMalloc(&b.d, v) == cudaSuccess &&
              cudaMalloc((void **)&b.SY, sizeof(double) * m * m) == cudaSuccess &&
              cudaMalloc((void **)&b.YY, sizeof(double) * m * m) == cudaSuccess &&
              cudaMalloc((void **)&b.part, sizeof(double) * nblk * (3 * m + 4)) == cudaSuccess &&
              cudaMalloc((void **)&b.coef, sizeof(double) * 2 * m) == cudaSuccess &&
              cudaMalloc((void **)&b.scal, sizeof(double) * 16) == cudaSuccess &&
              cudaMallocHost((void **)&b.scal_h, sizeof(double) * 16) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        solver_free(b);
        b.npix = npix;
        b.nblk = nblk;
        return IVIS_ERR_OOM;
    }
    cudaMemset(b.scal, 0, sizeof(double) * 16);
    return IVIS_OK;
}

__device__ __forceinline__ double block_max(double v, double *scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? scratch[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    }
    return s;
}

template <typename T>
__device__ __forceinline__ bool is_free(T x, T g, int pos) {
    return !(pos && x <= (T)0 && g > (T)0);
}

// x <- max(x, 0) when positivity is on.
template <typename T>
__global__ void k_sol_project(T *x, size_t n, int pos) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pos && x[i] < (T)0) x[i] = (T)0;
}

// Per CTA: a_t = s_t . g_F, b_t = y_t . g_F (chronological t), g_F . g_F and the projected-
// gradient infinity norm. part layout per CTA: [a(m) | b(m) | gg | pg].
template <typename T>
__global__ void __launch_bounds__(256)
k_sol_dots(size_t n, const T *__restrict__ x, const T *__restrict__ g, int pos,
           const T *__restrict__ S, const T *__restrict__ Y, SlotList ord, int stride,
           double *part) {
    __shared__ T gf[SOL_CHUNK];
    __shared__ double red[32];
    const size_t base = (size_t)blockIdx.x * SOL_CHUNK;
    double gg = 0.0;
    T pg = (T)0;
    for (int i = threadIdx.x; i < SOL_CHUNK; i += blockDim.x) {
        const size_t idx = base + i;
        T v = (T)0;
        if (idx < n) {
            const T xi = x[idx], gi = g[idx];
            v = is_free(xi, gi, pos) ? gi : (T)0;
            const T pgi = pos ? fabs(fmax(xi - gi, (T)0) - xi) : fabs(gi);
            pg = fmax(pg, pgi);
            gg = fma((double)v, (double)v, gg);
        }
        gf[i] = v;
    }
    __syncthreads();
    double *out = part + (size_t)blockIdx.x * stride;
    for (int t = 0; t < 2 * ord.m; ++t) {
        const T *vec = (t < ord.m ? S : Y) + (size_t)ord.slot[t < ord.m ? t : t - ord.m] * n;
        double acc = 0.0;
        for (int i = threadIdx.x; i < SOL_CHUNK; i += blockDim.x) {
            const size_t idx = base + i;
            if (idx < n) acc = fma((double)vec[idx], (double)gf[i], acc);
        }
        const double sum = block_sum(acc, red);
        if (threadIdx.x == 0) out[t] = sum;
    }
    const double ggs = block_sum(gg, red);
    if (threadIdx.x == 0) out[2 * ord.m] = ggs;
    const double pgm = block_max((double)pg, red);
    if (threadIdx.x == 0) out[2 * ord.m + 1] = pgm;
}

// Sum the per-CTA partials (fixed order) and form the compact-representation coefficients.
// scal: [0] gamma (kept between iterations), [2] pg_inf, [3] g_F.g_F.
__global__ void k_sol_small(int nblk, int stride, const double *__restrict__ part, SlotList ord,
                            const double *__restrict__ SY, const double *__restrict__ YY, int mcap,
                            double *coef, double *scal) {
    __shared__ double sums[2 * SOL_MAXM + 2];
    const int nd = 2 * ord.m + 2;
    // one warp per sum: lanes stride over the CTA partials, then a fixed shuffle tree
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int t = threadIdx.x >> 5; t < nd; t += nw) {
        const bool mx = t == 2 * ord.m + 1;
        double acc = 0.0;
        for (int b = lane; b < nblk; b += 32) {
            const double v = part[(size_t)b * stride + t];
            acc = mx ? fmax(acc, v) : acc + v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = mx ? fmax(acc, u) : acc + u;
        }
        if (lane == 0) sums[t] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int m = ord.m;
    scal[2] = sums[2 * m + 1];
    scal[3] = sums[2 * m];
    if (m == 0) return;
    const double gamma = scal[0];
    double a[SOL_MAXM], b[SOL_MAXM], t[SOL_MAXM], w[SOL_MAXM], p1[SOL_MAXM];
    for (int i = 0; i < m; ++i) { a[i] = sums[i]; b[i] = sums[m + i]; }
    // R[i][j] = s_i . y_j (i <= j), chronological order
    auto R = [&](int i, int j) { return SY[ord.slot[i] * mcap + ord.slot[j]]; };
    for (int i = m - 1; i >= 0; --i) {  // t = R^{-1} a
        double acc = a[i];
        for (int j = i + 1; j < m; ++j) acc -= R(i, j) * t[j];
        t[i] = acc / R(i, i);
    }
    for (int i = 0; i < m; ++i) {  // w = (D + gamma Y^T Y) t - gamma b
        double acc = R(i, i) * t[i];
        for (int j = 0; j < m; ++j) acc += gamma * YY[ord.slot[i] * mcap + ord.slot[j]] * t[j];
        w[i] = acc - gamma * b[i];
    }
    for (int i = 0; i < m; ++i) {  // p1 = R^{-T} w
        double acc = w[i];
        for (int j = 0; j < i; ++j) acc -= R(j, i) * p1[j];
        p1[i] = acc / R(i, i);
    }
    for (int i = 0; i < m; ++i) {
        coef[i] = p1[i];
        coef[m + i] = -gamma * t[i];
    }
}

// d = -[ gamma g_F + S coef_s + Y coef_y ] on F, 0 elsewhere (m == 0: d = -g_F).
// part per CTA: [g.d] at offset 0.
template <typename T>
__global__ void __launch_bounds__(256)
k_sol_dir(size_t n, const T *__restrict__ x, const T *__restrict__ g, int pos,
          const T *__restrict__ S, const T *__restrict__ Y, SlotList ord,
          const double *__restrict__ coef, const double *__restrict__ scal, T *d, int stride,
          double *part) {
    __shared__ double red[32];
    __shared__ T cf[2 * SOL_MAXM];
    const size_t base = (size_t)blockIdx.x * SOL_CHUNK;
    const T gamma = ord.m ? (T)scal[0] : (T)1;
    for (int t = threadIdx.x; t < 2 * ord.m; t += blockDim.x) cf[t] = (T)coef[t];
    __syncthreads();
    double gd = 0.0;  // d is stored in the working precision; so is its per-pixel arithmetic
    for (int i = threadIdx.x; i < SOL_CHUNK; i += blockDim.x) {
        const size_t idx = base + i;
        if (idx >= n) continue;
        const T xi = x[idx], gi = g[idx];
        T dv = (T)0;
        if (is_free(xi, gi, pos)) {
            T acc = gamma * gi;
            for (int t = 0; t < ord.m; ++t) {
                acc += cf[t] * S[(size_t)ord.slot[t] * n + idx];
                acc += cf[ord.m + t] * Y[(size_t)ord.slot[t] * n + idx];
            }
            dv = -acc;
        }
        d[idx] = dv;
        gd = fma((double)gi, (double)dv, gd);
    }
    const double gds = block_sum(gd, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * stride] = gds;
}

// scal[slot_out] = sum of part[b * stride] over CTAs (fixed order).
__global__ void k_sol_sum(int nblk, int stride, const double *__restrict__ part, double *scal,
                          int slot_out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(size_t)b * stride];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) scal[slot_out] = acc;
}

// Trial point x = P(xk + alpha d); part per CTA: [gk . (x - xk)].
template <typename T>
__global__ void __launch_bounds__(256)
k_sol_trial(size_t n, const T *__restrict__ xk, const T *__restrict__ gk, const T *__restrict__ d,
            double alpha, int pos, T *x, int stride, double *part) {
    __shared__ double red[32];
    const size_t base = (size_t)blockIdx.x * SOL_CHUNK;
    const T al = (T)alpha;
    double acc = 0.0;
    for (int i = threadIdx.x; i < SOL_CHUNK; i += blockDim.x) {
        const size_t idx = base + i;
        if (idx >= n) continue;
        const T xo = xk[idx];
        T v = xo + al * d[idx];
        if (pos && v < (T)0) v = (T)0;
        x[idx] = v;
        acc = fma((double)gk[idx], (double)(v - xo), acc);
    }
    const double sum = block_sum(acc, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * stride] = sum;
}

// New correction pair into slot `slot`: s = x - xk, y = g - gk; xk <- x, gk <- g. Per CTA
// partials of s.y_t, s_t.y, y.y_t for every slot t of `ord` (which ends with `slot`).
template <typename T>
__global__ void __launch_bounds__(256)
k_sol_update(size_t n, const T *__restrict__ x, const T *__restrict__ g, T *xk, T *gk, T *S, T *Y,
             int slot, SlotList ord, int stride, double *part) {
    __shared__ T sv[SOL_CHUNK], yv[SOL_CHUNK];
    __shared__ double red[32];
    const size_t base = (size_t)blockIdx.x * SOL_CHUNK;
    for (int i = threadIdx.x; i < SOL_CHUNK; i += blockDim.x) {
        const size_t idx = base + i;
        T s = (T)0, y = (T)0;
        if (idx < n) {
            const T xi = x[idx], gi = g[idx];
            s = xi - xk[idx];
            y = gi - gk[idx];
            S[(size_t)slot * n + idx] = s;
            Y[(size_t)slot * n + idx] = y;
            xk[idx] = xi;
            gk[idx] = gi;
        }
        sv[i] = s;
        yv[i] = y;
    }
    __syncthreads();
    double *out = part + (size_t)blockIdx.x * stride;
    for (int t = 0; t < ord.m; ++t) {
        const int st = ord.slot[t];
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = threadIdx.x; i < SOL_CHUNK; i += blockDim.x) {
            const size_t idx = base + i;
            if (idx >= n) continue;
            const T ys = st == slot ? yv[i] : Y[(size_t)st * n + idx];
            const T ss = st == slot ? sv[i] : S[(size_t)st * n + idx];
            a = fma((double)sv[i], (double)ys, a);
            b = fma((double)ss, (double)yv[i], b);
            c = fma((double)yv[i], (double)ys, c);
        }
        const double as = block_sum(a, red);
        const double bs = block_sum(b, red);
        const double cs = block_sum(c, red);
        if (threadIdx.x == 0) {
            out[3 * t] = as;
            out[3 * t + 1] = bs;
            out[3 * t + 2] = cs;
        }
    }
}

// Accept the pair if s.y > eps y.y: fill SY/YY rows and columns of `slot`, gamma = s.y / y.y.
// scal: [5] accepted flag, [6] s.y, [7] y.y.
__global__ void k_sol_update_small(int nblk, int stride, const double *__restrict__ part,
                                   int slot, SlotList ord, double *SY, double *YY, int mcap,
                                   double eps, double *scal) {
    __shared__ double sums[3 * SOL_MAXM];
    const int nd = 3 * ord.m;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int t = threadIdx.x >> 5; t < nd; t += nw) {  // one warp per sum, fixed order
        double acc = 0.0;
        for (int b = lane; b < nblk; b += 32) acc += part[(size_t)b * stride + t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) sums[t] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int self = -1;
    for (int t = 0; t < ord.m; ++t)
        if (ord.slot[t] == slot) self = t;
    const double sy = self >= 0 ? sums[3 * self] : 0.0;
    const double yy = self >= 0 ? sums[3 * self + 2] : 0.0;
    scal[6] = sy;
    scal[7] = yy;
    const bool ok = sy > eps * yy && yy > 0.0;
    scal[5] = ok ? 1.0 : 0.0;
    if (!ok) return;
    for (int t = 0; t < ord.m; ++t) {
        const int st = ord.slot[t];
        SY[slot * mcap + st] = sums[3 * t];      // s_new . y_t
        SY[st * mcap + slot] = sums[3 * t + 1];  // s_t . y_new
        YY[slot * mcap + st] = sums[3 * t + 2];
        YY[st * mcap + slot] = sums[3 * t + 2];
    }
    scal[0] = sy / yy;
}

}  // namespace ivis
