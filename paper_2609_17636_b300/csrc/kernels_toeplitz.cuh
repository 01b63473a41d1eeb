// kernels_toeplitz.cuh -- the data term through the Toeplitz form of its normal operator.
//
// For one (pointing, channel) pair the window is z = A .* P x (nb x nb, Eq. 2) and the model
// visibilities are F z with F[j, p] = exp(-2 pi i u_j . l_p) (Eqs. 3-5). The data term of
// Eq. 6 and its window gradient expand to
//     Q = 1/2 z^T Re(H) z - z^T b + C,      dQ/dz = Re(H) z - b,
// with H = F^H W F, b = Re(F^H W V) and C = 1/2 sum_j w_j |V_j|^2. H[p, q] = T(l_p - l_q),
// T(d) = sum_j w_j exp(+2 pi i u_j . d), depends on the pixel difference only, d in (-nb, nb)^2:
// Re(H) z is a linear convolution of z with Re T, which a cyclic convolution of period
// nf = 2 nb reproduces exactly on the window. Re T is real and even, so its nf x nf DFT (That)
// is real and even, and
//     Re(H) z = crop_nb( IDFT( That .* DFT(pad_nf(z)) ) ) / nf^2.
// T and b are computed once per data set (adjoint NUFFTs on a 2 nb window); an evaluation then
// costs two pruned FFT passes per pair and no pass over the visibilities.
//
// Layouts: window pixel p sits at fine-grid index (p - nb/2) mod nf (as in the NUFFT passes);
// That is stored transposed, [slot][kx][ky], so that a column CTA reads it contiguously.
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "kernels_nufft.cuh"

namespace ivis {

// ----------------------------------------------------------------- set-up (once per pair)
// Rows of the cyclic kernel from the 2nb x 2nb window of offsets d = p' - nb (twin, scaled
// by sgn): T_emb[i][j] = Re T(d) at d = i, j folded to (-nb, nb); the row and column at
// d = -nb are never reached by a difference of two window pixels and are set to zero (which
// keeps the embedded kernel even). Each line is then DFT'ed along x.
template <typename T>
__global__ void __launch_bounds__(256)
k_toep_embed_rows(const T *__restrict__ twin, T sgn, typename cplx_of<T>::type *buf, int lognf,
                  const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, nb = nf >> 1, tpl = nf >> 4, lpb = blockDim.x / tpl;
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int i = blockIdx.x * lpb + l;
    const bool on = i < nf;  // small grids: fewer lines than the CTA holds
    const int si = (i + nb) & (nf - 1);
    for (int j = j0; j < nf; j += tpl) {
        const int sj = (j + nb) & (nf - 1);
        const T v = (!on || si == 0 || sj == 0) ? (T)0 : sgn * twin[(size_t)si * nf + sj];
        s[pidx(l * nf + j)] = mk(v, (T)0);
    }
    __syncthreads();
    line_fft<C, -1>(s, 1, l * nf, lognf, j0, tw);
    if (!on) return;
    C *out = buf + (size_t)i * nf;
    for (int j = j0; j < nf; j += tpl) out[j] = s[pidx(l * nf + j)];
}

// Column DFTs of the row-transformed kernel; keeps the real part times scale, transposed.
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_toep_embed_cols(const typename cplx_of<T>::type *__restrict__ buf, T *that_t, int lognf, int logc,
                  T scale, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, ncol = 1 << logc, tpl = nf >> 4;
    const int c0 = blockIdx.x << logc;
    const int c = threadIdx.x & (ncol - 1), j0 = threadIdx.x >> logc;
    for (int e = j0; e < nf; e += tpl) s[pidx((e << logc) + c)] = buf[(size_t)e * nf + c0 + c];
    __syncthreads();
    line_fft<C, -1>(s, ncol, c, lognf, j0, tw);
    for (int idx = threadIdx.x; idx < (nf << logc); idx += blockDim.x) {
        const int cc = idx >> lognf, e = idx & (nf - 1);
        that_t[(size_t)(c0 + cc) * nf + e] = s[pidx((e << logc) + cc)].x * scale;
    }
}

// b window from the centre of the 2nb window (scaled by sgn).
template <typename T>
__global__ void k_toep_crop(const T *__restrict__ win2, T sgn, T *bwin, int nb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nb) return;
    const int q = i / nb, p = i - q * nb;
    bwin[i] = sgn * win2[(size_t)(q + nb / 2) * (2 * nb) + p + nb / 2];
}

// FP64 partial sums of w |V|^2 over caller-order visibilities (float pairs).
__global__ void k_vis_energy(int m, const float *__restrict__ vis, const float *__restrict__ w,
                             double *part) {
    __shared__ double red[32];
    double a = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const double re = vis[2 * (size_t)j], im = vis[2 * (size_t)j + 1];
        a += (double)w[j] * (re * re + im * im);
    }
    a = block_sum(a, red);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

template <typename T>
__global__ void k_fill(size_t n, T v, T *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

__global__ void k_unit_vis(int m, float2 *v) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) v[j] = make_float2(1.0f, 0.0f);
}

// The per-evaluation passes (two slots per transform) are k_fwd_rows_pk, k_toep_cols_pk and
// k_toep_rows_pk in kernels_packed.cuh.

}  // namespace ivis
