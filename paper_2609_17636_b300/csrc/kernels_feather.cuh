// kernels_feather.cuh -- short-spacing correction by feathering (the paper's appendix).
//
//     I_comb = IDFT[ B DFT(s I_SD) + (1 - B) DFT(I_int) ] = I_int + IDFT[ B DFT(s I_SD - I_int) ]
//
// on the n x n image grid, B(k) = exp(-2 pi^2 sigma^2 |k|^2) = b1(kx) b1(ky) with b1 a 1D
// Gaussian of the frequency index. B is separable and real-even, so the correction is a
// circular convolution along x followed by one along y, each done per line as DFT, product
// with b1, inverse DFT in shared memory. Two real lines travel in one complex line (the
// filter is real and even, so the real and imaginary parts never mix).
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace ivis {

// Rows: line l of the CTA carries image rows 2r and 2r + 1 (r = blockIdx.x * lpb + l) of
// d = s * sd - int; writes the x-filtered d into out.
template <typename T>
__global__ void __launch_bounds__(256)
k_feather_rows(const T *__restrict__ i_int, const float *__restrict__ i_sd, T scale,
               const T *__restrict__ b1, T *out, int n, int logn,
               const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int tpl = n >> 4, lpb = blockDim.x / tpl;
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int r = blockIdx.x * lpb + l;
    const bool on = 2 * r < n;
    const size_t base = ((size_t)blockIdx.y * n + 2 * (size_t)r) * n;
    for (int j = j0; j < n; j += tpl) {
        C v = mk((T)0, (T)0);
        if (on) {
            v.x = scale * (T)i_sd[base + j] - i_int[base + j];
            v.y = scale * (T)i_sd[base + n + j] - i_int[base + n + j];
        }
        s[pidx(l * n + j)] = v;
    }
    __syncthreads();
    line_fft<C, -1>(s, 1, l * n, logn, j0, tw);
    for (int j = j0; j < n; j += tpl) {
        C &v = s[pidx(l * n + j)];
        const T b = b1[j];
        v = mk(v.x * b, v.y * b);
    }
    __syncthreads();
    line_fft<C, +1>(s, 1, l * n, logn, j0, tw);
    if (!on) return;
    const T inv = (T)1 / (T)n;
    for (int j = j0; j < n; j += tpl) {
        const C v = s[pidx(l * n + j)];
        out[base + j] = v.x * inv;
        out[base + n + j] = v.y * inv;
    }
}

// Columns: a CTA owns 2 * ncol adjacent columns; complex line c carries columns c0 + c and
// c0 + ncol + c. Filters along y in place and adds the interferometric map.
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_feather_cols(const T *__restrict__ i_int, const T *__restrict__ b1, T *out, int n, int logn,
               int logc, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int ncol = 1 << logc, tpl = n >> 4;
    const int c0 = blockIdx.x * 2 * ncol;
    const int c = threadIdx.x & (ncol - 1), j0 = threadIdx.x >> logc;
    const size_t img = (size_t)blockIdx.y * n * n;
    for (int e = j0; e < n; e += tpl)
        s[pidx((e << logc) + c)] = mk(out[img + (size_t)e * n + c0 + c], out[img + (size_t)e * n + c0 + ncol + c]);
    __syncthreads();
    line_fft<C, -1>(s, ncol, c, logn, j0, tw);
    for (int e = j0; e < n; e += tpl) {
        C &v = s[pidx((e << logc) + c)];
        const T b = b1[e];
        v = mk(v.x * b, v.y * b);
    }
    __syncthreads();
    line_fft<C, +1>(s, ncol, c, logn, j0, tw);
    const T inv = (T)1 / (T)n;
    for (int e = j0; e < n; e += tpl) {
        const C v = s[pidx((e << logc) + c)];
        const size_t i0 = img + (size_t)e * n + c0 + c, i1 = i0 + ncol;
        out[i0] = i_int[i0] + v.x * inv;
        out[i1] = i_int[i1] + v.y * inv;
    }
}

}  // namespace ivis
