// kernels_sdconv.cuh -- the dish-beam convolution of the fusion term (Eqs. 11-13) through
// line DFTs.
//
// B (x) I is separable with the same symmetric taps b[-R..R] along x and y, truncated at
// R = ceil(4 sigma_B) and zero outside the image. Along one axis, a cyclic convolution of
// period N >= n + R of the zero-padded line reproduces the linear one on [0, n) exactly (no
// wrapped index lands inside the image), so each pass is: line DFT, product with the taps'
// spectrum spec[k] = (b[0] + 2 sum_{t>=1} b[t] cos(2 pi k t / N)) / N (real and even), inverse
// DFT, crop. Two real lines share one complex line (the real-even filter keeps the real and
// imaginary parts apart). The column pass can fuse the single-dish residual
// e = (t - T) / sigma^2, the per-CTA partials of K = 1/2 sum (t - T)^2 / sigma^2 and the first
// pass of the gradient B^T e: the taps are symmetric (B^T = B) and the two axes' passes
// commute, so the column pass convolves e along its column at once and one row pass finishes
// the gradient (three launches in all instead of four).
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace ivis {

// Rows: line l of the CTA carries image rows 2r and 2r + 1 of channel blockIdx.y
// (r = blockIdx.x * lpb + l). CTA = lpb lines of N/16 threads.
template <typename T>
__global__ void __launch_bounds__(512)
k_sdconv_rows(const T *__restrict__ in, T *out, const T *__restrict__ spec, int n, int logN,
              const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int N = 1 << logN, tpl = N >> 4, lpb = blockDim.x / tpl;
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int r = blockIdx.x * lpb + l, c = blockIdx.y;
    const bool on = 2 * r < n;
    const size_t base = ((size_t)c * n + 2 * (size_t)r) * n;
    const T *sp = spec + (size_t)c * N;
    for (int j = j0; j < N; j += tpl) {
        C v = mk((T)0, (T)0);
        if (on && j < n) v = mk(in[base + j], 2 * r + 1 < n ? in[base + n + j] : (T)0);
        s[pidx(l * N + j)] = v;
    }
    __syncthreads();
    line_fft<C, -1>(s, 1, l * N, logN, j0, tw);
    for (int j = j0; j < N; j += tpl) {
        C &v = s[pidx(l * N + j)];
        const T b = sp[j];
        v = mk(v.x * b, v.y * b);
    }
    __syncthreads();
    line_fft<C, +1>(s, 1, l * N, logN, j0, tw);
    if (!on) return;
    for (int j = j0; j < n; j += tpl) {
        const C v = s[pidx(l * N + j)];
        out[base + j] = v.x;
        if (2 * r + 1 < n) out[base + n + j] = v.y;
    }
}

// Columns: a CTA owns 2 * ncol adjacent columns of channel blockIdx.y; complex line q carries
// columns x0 + q and x0 + ncol + q. FUSED: with e = (t - tsd) * inv_sig2[c], out = the column
// convolution of e, and this CTA's share of K to kpart[c * gridDim.x + blockIdx.x].
template <typename T, int FUSED>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_sdconv_cols(const T *__restrict__ in, T *out, const T *__restrict__ spec, int n, int logN, int logc,
              const typename cplx_of<T>::type *__restrict__ tw, const T *__restrict__ tsd,
              const double *__restrict__ inv_sig2, double *kpart) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    __shared__ double red[32];
    const int N = 1 << logN, ncol = 1 << logc, tpl = N >> 4;
    const int x0 = blockIdx.x * 2 * ncol, c = blockIdx.y;
    const int q = threadIdx.x & (ncol - 1), j0 = threadIdx.x >> logc;
    const size_t img = (size_t)c * n * n;
    const int xa = x0 + q, xb = x0 + ncol + q;
    const T *sp = spec + (size_t)c * N;
    for (int e = j0; e < N; e += tpl) {
        C v = mk((T)0, (T)0);
        if (e < n) v = mk(xa < n ? in[img + (size_t)e * n + xa] : (T)0, xb < n ? in[img + (size_t)e * n + xb] : (T)0);
        s[pidx((e << logc) + q)] = v;
    }
    __syncthreads();
    line_fft<C, -1>(s, ncol, q, logN, j0, tw);
    for (int e = j0; e < N; e += tpl) {
        C &v = s[pidx((e << logc) + q)];
        const T b = sp[e];
        v = mk(v.x * b, v.y * b);
    }
    __syncthreads();
    line_fft<C, +1>(s, ncol, q, logN, j0, tw);
    if (FUSED) {
        // e in place of t (zero outside the image: the padding of the second convolution)
        T kloc = (T)0;  // at most 2 n / tpl terms per thread in the working precision, then FP64
        const T is2 = (T)inv_sig2[c];
        for (int e = j0; e < N; e += tpl) {
            C &v = s[pidx((e << logc) + q)];
            C o = mk((T)0, (T)0);
            if (e < n) {
                const size_t ia = img + (size_t)e * n + xa, ib = img + (size_t)e * n + xb;
                if (xa < n) {
                    const T d = v.x - tsd[ia];
                    kloc += (T)0.5 * d * d * is2;
                    o.x = d * is2;
                }
                if (xb < n) {
                    const T d = v.y - tsd[ib];
                    kloc += (T)0.5 * d * d * is2;
                    o.y = d * is2;
                }
            }
            v = o;
        }
        __syncthreads();
        line_fft<C, -1>(s, ncol, q, logN, j0, tw);
        for (int e = j0; e < N; e += tpl) {
            C &v = s[pidx((e << logc) + q)];
            const T b = sp[e];
            v = mk(v.x * b, v.y * b);
        }
        __syncthreads();
        line_fft<C, +1>(s, ncol, q, logN, j0, tw);
        const double ks = block_sum((double)kloc, red);
        if (threadIdx.x == 0) kpart[(size_t)c * gridDim.x + blockIdx.x] = ks;
    }
    for (int e = j0; e < n; e += tpl) {
        const C v = s[pidx((e << logc) + q)];
        const size_t ia = img + (size_t)e * n + xa, ib = img + (size_t)e * n + xb;
        if (xa < n) out[ia] = v.x;
        if (xb < n) out[ib] = v.y;
    }
}

}  // namespace ivis
