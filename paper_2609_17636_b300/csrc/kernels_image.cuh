// kernels_image.cuh -- image-domain terms and the cost reductions.
//
//   a6  joint sum over pointings of the per-pointing adjoint images (Eq. 6), deterministic
//       order, + lambda_r grad R + lambda_s grad K                         (k_assemble)
//   a7  Laplacian regulariser R = 1/2 ||D I||^2, grad R = D^T D I (Eqs. 7-8), zero
//       boundary, evaluated on the fly in k_assemble
//   a8  fusion term: t = B (x) I by two separable passes, e = (t - T)/sigma^2,
//       K = 1/2 sum (t - T)^2 / sigma^2, grad K = B (x) e (Eqs. 11-13)  (k_conv_rows/cols)
//   a9  Q_tot = Q + lambda_s K + lambda_r R from FP64 partials in a fixed order (k_finalize)
#pragma once
#include "common.cuh"
#include "kernels_nufft.cuh"

namespace ivis {

template <typename T>
__device__ __forceinline__ T pix(const T *__restrict__ I, int n, int y, int x) {
    return (y >= 0 && y < n && x >= 0 && x < n) ? I[(size_t)y * n + x] : (T)0;
}
template <typename T>
__device__ __forceinline__ T lap(const T *__restrict__ I, int n, int y, int x) {
    return (T)4 * pix(I, n, y, x) - pix(I, n, y - 1, x) - pix(I, n, y + 1, x) -
           pix(I, n, y, x - 1) - pix(I, n, y, x + 1);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_assemble(const T *__restrict__ sky, const T *__restrict__ contrib,
           const PairInfo *__restrict__ pinfo, const int *__restrict__ chan_start,
           const int *__restrict__ chan_list, const T *__restrict__ gradK, T *grad, int n, int nb,
           int nchan, T lr, T ls, int use_r, int use_k, double *rpart) {
    __shared__ double red[32];
    const size_t npix = (size_t)n * n;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rloc = 0.0;
    if (idx < npix * nchan) {
        const int chan = (int)(idx / npix);
        const int rem = (int)(idx - (size_t)chan * npix);
        const int y = rem / n, x = rem - y * n;
        T g = (T)0;
        for (int t = chan_start[chan]; t < chan_start[chan + 1]; ++t) {
            const int slot = chan_list[t];
            const PairInfo pi = pinfo[slot];
            const int q = y - (pi.cy - nb / 2), p = x - (pi.cx - nb / 2);
            if ((unsigned)q < (unsigned)nb && (unsigned)p < (unsigned)nb)
                g += contrib[((size_t)slot * nb + q) * nb + p];
        }
        if (use_r) {
            const T *I = sky + (size_t)chan * npix;
            const T d0 = lap(I, n, y, x);
            T gr = (T)4 * d0;
            if (y > 0) gr -= lap(I, n, y - 1, x);
            if (y < n - 1) gr -= lap(I, n, y + 1, x);
            if (x > 0) gr -= lap(I, n, y, x - 1);
            if (x < n - 1) gr -= lap(I, n, y, x + 1);
            g += lr * gr;
            rloc = 0.5 * (double)d0 * (double)d0;
        }
        if (use_k) g += ls * gradK[idx];
        grad[idx] = g;
    }
    const double s = block_sum(rloc, red);
    if (threadIdx.x == 0) rpart[blockIdx.x] = s;
}

// out[c][y][x] = sum_{t=-R..R} b_c[t] in[c][y][x - t], zero outside; block = 256 outputs of a row.
template <typename T>
__global__ void __launch_bounds__(256)
k_conv_rows(const T *__restrict__ in, T *out, const T *__restrict__ taps, int R, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sh = reinterpret_cast<T *>(smem_raw);
    const int x0 = blockIdx.x * 256, y = blockIdx.y, c = blockIdx.z;
    const T *row = in + ((size_t)c * n + y) * n;
    const T *b = taps + (size_t)c * (2 * R + 1);
    for (int i = threadIdx.x; i < 256 + 2 * R; i += 256) {
        const int x = x0 - R + i;
        sh[i] = (x >= 0 && x < n) ? row[x] : (T)0;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= n) return;
    T acc = (T)0;
    const T *s = sh + threadIdx.x + 2 * R;
    for (int t = 0; t <= 2 * R; ++t) acc += __ldg(&b[t]) * s[-t];
    out[((size_t)c * n + y) * n + x] = acc;
}

// Column pass; block (32, 8) covers 32 columns x TY output rows. FUSED: the output is the
// single-dish residual e = (t - T)/sigma^2 and the block's share of K is written to kpart.
template <typename T, int FUSED>
__global__ void __launch_bounds__(256)
k_conv_cols(const T *__restrict__ in, T *out, const T *__restrict__ taps, int R, int n, int TY,
            const T *__restrict__ tsd, const double *__restrict__ inv_sig2, double *kpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    T *sh = reinterpret_cast<T *>(smem_raw);
    const int tx = threadIdx.x & 31, tyi = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + tx, y0 = blockIdx.y * TY, c = blockIdx.z;
    const T *img = in + (size_t)c * n * n;
    const T *b = taps + (size_t)c * (2 * R + 1);
    for (int i = tyi; i < TY + 2 * R; i += 8) {
        const int y = y0 - R + i;
        sh[i * 32 + tx] = (y >= 0 && y < n && x < n) ? img[(size_t)y * n + x] : (T)0;
    }
    __syncthreads();
    double kloc = 0.0;
    const double is2 = FUSED ? inv_sig2[c] : 0.0;
    for (int yy = tyi; yy < TY; yy += 8) {
        const int y = y0 + yy;
        if (y >= n || x >= n) continue;
        T acc = (T)0;
        const T *s = sh + (yy + 2 * R) * 32 + tx;
        for (int t = 0; t <= 2 * R; ++t) acc += __ldg(&b[t]) * s[-t * 32];
        const size_t o = ((size_t)c * n + y) * n + x;
        if (FUSED) {
            const double e = (double)acc - (double)tsd[o];
            kloc += 0.5 * e * e * is2;
            out[o] = (T)(e * is2);
        } else {
            out[o] = acc;
        }
    }
    if (FUSED) {
        const double s = block_sum(kloc, red);
        if (threadIdx.x == 0)
            kpart[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

// out = {Q_tot, Q, K, R}; fixed summation order (deterministic for a fixed launch shape).
__global__ void k_finalize(const double *__restrict__ jpart, int nj, const double *__restrict__ kpart,
                           int nk, const double *__restrict__ rpart, int nr, double lr, double ls,
                           double *out) {
    __shared__ double red[32];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nj; i += blockDim.x) a += jpart[i];
    for (int i = threadIdx.x; i < nk; i += blockDim.x) b += kpart[i];
    for (int i = threadIdx.x; i < nr; i += blockDim.x) c += rpart[i];
    const double Q = block_sum(a, red);
    const double K = block_sum(b, red);
    const double R = block_sum(c, red);
    if (threadIdx.x == 0) {
        out[1] = Q;
        out[2] = K;
        out[3] = R;
        out[0] = Q + ls * K + lr * R;
    }
}

template <typename T>
__global__ void k_f32_to(const float *__restrict__ in, T *out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}

}  // namespace ivis
