// kernels_image.cuh -- image-domain terms and the cost reductions.
//
//   a6  joint sum over pointings of the per-pointing adjoint images (Eq. 6), deterministic
//       order, + lambda_r grad R + lambda_s grad K                         (k_assemble)
//   a7  Laplacian regulariser R = 1/2 ||D I||^2, grad R = D^T D I (Eqs. 7-8), zero
//       boundary, evaluated on the fly in k_assemble
//   a8  fusion term: t = B (x) I by two separable passes, e = (t - T)/sigma^2,
//       K = 1/2 sum (t - T)^2 / sigma^2, grad K = B (x) e (Eqs. 11-13)  (k_conv_axis)
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

// Separable dish-beam convolution, one axis per launch: out = sum_{t=-R..R} b_c[t] in(. - t),
// zero outside the image. A CTA of 8 warps covers 32 lines (one per lane) x CONV_TO outputs
// along the convolution axis; each thread produces CONV_OPT consecutive outputs from a
// sliding window of registers, so each shared-memory load feeds CONV_OPT FMAs. The staged
// strip is laid out [position][line] with a 33-word row pitch (rows pass: lines are image
// rows and the transpose would otherwise serialise on one bank).
constexpr int CONV_OPT = 8;
constexpr int CONV_TO = 8 * CONV_OPT;  // outputs per CTA along the axis

// AXIS 0: along x (lines = rows); AXIS 1: along y (lines = columns).
// FUSED (AXIS 1 only): out = e = (t - T)/sigma^2 and the CTA's share of K goes to kpart.
template <typename T, int AXIS, int FUSED>
__global__ void __launch_bounds__(256)
k_conv_axis(const T *__restrict__ in, T *out, const T *__restrict__ taps, int R, int n,
            const T *__restrict__ tsd, const double *__restrict__ inv_sig2, double *kpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const int P = 33;
    const int L = CONV_TO + 2 * R;  // staged positions
    T *sh = reinterpret_cast<T *>(smem_raw);
    T *tp = sh + (size_t)L * P;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int line0 = blockIdx.x * 32, pos0 = blockIdx.y * CONV_TO, c = blockIdx.z;
    const T *img = in + (size_t)c * n * n;
    const T *b = taps + (size_t)c * (2 * R + 1);
    for (int t = threadIdx.x; t <= 2 * R; t += blockDim.x) tp[t] = b[t];
    if (AXIS == 0) {
        // rows: global reads run along x (positions) for coalescing
        for (int i = threadIdx.x; i < 32 * L; i += blockDim.x) {
            const int li = i / L, pi = i - li * L;
            const int y = line0 + li, x = pos0 - R + pi;
            sh[pi * P + li] = (y < n && x >= 0 && x < n) ? img[(size_t)y * n + x] : (T)0;
        }
    } else {
        for (int i = threadIdx.x; i < 32 * L; i += blockDim.x) {
            const int pi = i >> 5, li = i & 31;
            const int y = pos0 - R + pi, x = line0 + li;
            sh[pi * P + li] = (x < n && y >= 0 && y < n) ? img[(size_t)y * n + x] : (T)0;
        }
    }
    __syncthreads();
    // outputs j = 0..OPT-1 at axis position o0 + j use staged position o0 + j + 2R - t
    const int o0 = wid * CONV_OPT;
    T acc[CONV_OPT], win[CONV_OPT];
#pragma unroll
    for (int j = 0; j < CONV_OPT; ++j) {
        acc[j] = (T)0;
        win[j] = sh[(o0 + j + 2 * R) * P + lane];
    }
    for (int t = 0; t <= 2 * R; ++t) {
        const T bt = tp[t];
#pragma unroll
        for (int j = 0; j < CONV_OPT; ++j) acc[j] += bt * win[j];
        if (t < 2 * R) {
#pragma unroll
            for (int j = CONV_OPT - 1; j > 0; --j) win[j] = win[j - 1];
            win[0] = sh[(o0 + 2 * R - t - 1) * P + lane];
        }
    }
    double kloc = 0.0;
    const double is2 = FUSED ? inv_sig2[c] : 0.0;
    const int line = line0 + lane;
#pragma unroll
    for (int j = 0; j < CONV_OPT; ++j) {
        const int pos = pos0 + o0 + j;
        if (line >= n || pos >= n) continue;
        const size_t o = AXIS == 0 ? ((size_t)c * n + line) * n + pos : ((size_t)c * n + pos) * n + line;
        if (FUSED) {
            const double e = (double)acc[j] - (double)tsd[o];
            kloc += 0.5 * e * e * is2;
            out[o] = (T)(e * is2);
        } else {
            out[o] = acc[j];
        }
    }
    if (FUSED) {
        const double sum = block_sum(kloc, red);
        if (threadIdx.x == 0)
            kpart[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum;
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
