// kernels_wstack.cuh -- the w-term of the full visibility equation (Eq. 1) by w-stacking.
//
// Eq. 1 adds, per visibility j and window pixel p, the factor exp(-2 pi i w_j (n_p - 1)) / n_p
// (n = sqrt(1 - l^2 - m^2)). The phase is split as w_j x_c + w_j x'_p, x_c the centre of the
// window's range of n - 1, |x'_p| <= X. The remaining factor is interpolated between w-planes
// w_k = w0 + k dw with the same ES kernel phi as the uv gridding (a type-3 step along w; by
// Poisson summation the aliased terms are the kernel's transform Phi beyond 3/4 when dw X <= 1/4):
//     exp(-2 pi i w x') = sum_k phi((w - w_k)/dw) exp(-2 pi i w_k x') / Phi(dw x') + O(tol),
// so that
//     V~_j = exp(-2 pi i w_j x_c) sum_k phi_jk NUFFT2[ A I' corr exp(-2 pi i w_k x') ](u_j, v_j),
//     corr = 1 / (n Phi(dw x')).
// Each (pair, plane) is a slot of the 2D machinery (forward and adjoint FFT passes with the
// plane's modulation folded into the row passes); each visibility appears as W entries, one per
// plane of its kernel support, sorted per plane by tile and first-tap cell. An evaluation runs
// the grid pass twice over the entries: interpolation only (entry values by vis-major index),
// then, after the per-visibility residuals (this file), spreading only.
#pragma once
#include "common.cuh"
#include "kernels_nufft.cuh"

namespace ivis {

// Per-pair data of the residual / gather kernel (caller order of the pair's visibilities).
template <typename T> struct WPair {
    const typename cplx_of<T>::type *V;      // observed visibilities
    const T *w;                              // weights
    const typename cplx_of<T>::type *phase;  // exp(-2 pi i w_j x_c)
    const T *wk;                             // [m][W] w-kernel weights phi_jk
    const int *epos;                         // [m][W] sorted entry position of (j, t)
    typename cplx_of<T>::type *ent_val;      // sorted entry values (spread input)
    long long pv_off;                        // offset of the pair's [m][W] interpolated values
    int m;
};

// Per-CTA min and max of the w column (the host reduces the CTA results).
__global__ void k_w_minmax(int m, const float *__restrict__ uvw, float *mm) {
    __shared__ float lo[256], hi[256];
    float a = 3.0e38f, b = -3.0e38f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const float w = uvw[3 * (size_t)j + 2];
        a = fminf(a, w);
        b = fmaxf(b, w);
    }
    lo[threadIdx.x] = a;
    hi[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            lo[threadIdx.x] = fminf(lo[threadIdx.x], lo[threadIdx.x + o]);
            hi[threadIdx.x] = fmaxf(hi[threadIdx.x], hi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mm[2 * blockIdx.x] = lo[0];
        mm[2 * blockIdx.x + 1] = hi[0];
    }
}

// Expands each visibility into W entries: plane k = k0 + t with k0 = floor(a - W/2) + 1,
// a = (w - w0)/dw, weight phi(a - k); the entry key is the plane-major extension of the
// visibility's tile/cell key. Also the per-visibility phase exp(-2 pi i w x_c), V and w in
// the working precision (caller order).
template <typename T>
__global__ void k_w_entries(int m, int W, int nplane, const float *__restrict__ uvw, const float *__restrict__ vis,
                            const float *__restrict__ wt, double w0, double dw, double xc, double beta,
                            long long nf2, const typename coord_of<T>::type *__restrict__ coord_tmp,
                            const int *__restrict__ key, typename coord_of<T>::type *coord_e,
                            int *key_e, T *wk, typename cplx_of<T>::type *phase,
                            typename cplx_of<T>::type *vout, T *wout, int *err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double w = (double)uvw[3 * (size_t)j + 2];
    if (!isfinite(w)) {
        atomicOr(err, 1);
        w = w0;
    }
    const double a = (w - w0) / dw;
    // the plane range covers every finite w with half a plane to spare; the clamp only
    // guards the keys (and thus the sort's counters) against rounding at the ends
    const int k0 = min(max((int)floor(a - 0.5 * W) + 1, 0), nplane - W);
    for (int t = 0; t < W; ++t) {
        const size_t i = (size_t)j * W + t;
        const int k = k0 + t;
        coord_e[i] = coord_tmp[j];
        key_e[i] = (int)((long long)k * nf2 + key[j]);
        wk[i] = (T)es_kernel((a - (double)k) * 2.0 / (double)W, beta);
    }
    double s, c;
    sincospi(-2.0 * w * xc, &s, &c);
    phase[j] = mk((T)c, (T)s);
    vout[j] = mk((T)vis[2 * (size_t)j], (T)vis[2 * (size_t)j + 1]);
    wout[j] = (T)wt[j];
}

// Scatter of the entries into key order; epos[i] = the entry's sorted position.
template <typename T>
__global__ void k_w_scatter(long long E, const int *__restrict__ key_e,
                            const typename coord_of<T>::type *__restrict__ coord_e,
                            const T *__restrict__ wk, int *cursor, typename coord_of<T>::type *coord,
                            T *w_sorted, int *orig, int *epos) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E) return;
    const int pos = atomicAdd(&cursor[key_e[i]], 1);
    coord[pos] = coord_e[i];
    w_sorted[pos] = wk[i];
    orig[pos] = (int)i;
    epos[i] = pos;
}

// Per visibility: V~ = phase sum_t phi_t pv[t]. PREDICT: V~ to out (caller order). Otherwise
// r = V~ - V, the CTA's partial of 1/2 w |r|^2 (FP64 across warps) to jpart[pair * gridDim.x + blockIdx.x], and
// the spread value w r conj(phase) to the visibility's W entries.
template <typename T, bool PREDICT>
__global__ void __launch_bounds__(256)
k_w_residual(const WPair<T> *__restrict__ wpairs, int W, const typename cplx_of<T>::type *__restrict__ pv,
             double *jpart, typename cplx_of<T>::type *out) {
    typedef typename cplx_of<T>::type C;
    __shared__ double red[32];
    const WPair<T> wp = wpairs[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    T jacc = (T)0;
    if (j < wp.m) {
        const C *pj = pv + wp.pv_off + (size_t)j * W;
        const T *kj = wp.wk + (size_t)j * W;
        C s = mk((T)0, (T)0);
        for (int t = 0; t < W; ++t) {
            const C v = pj[t];
            const T k = kj[t];
            s.x += k * v.x;
            s.y += k * v.y;
        }
        const C vt = cmul(s, wp.phase[j]);
        if (PREDICT) {
            out[j] = vt;
        } else {
            const C V = wp.V[j];
            const T w = wp.w[j];
            const C r = mk(vt.x - V.x, vt.y - V.y);
            jacc = (T)0.5 * w * (r.x * r.x + r.y * r.y);
            const C c = cmulc(mk(w * r.x, w * r.y), wp.phase[j]);
            const int *ej = wp.epos + (size_t)j * W;
            for (int t = 0; t < W; ++t) wp.ent_val[ej[t]] = c;
        }
    }
    if (PREDICT) return;
    const double js = block_sum_t(jacc, red);
    if (threadIdx.x == 0) jpart[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = js;
}

}  // namespace ivis
