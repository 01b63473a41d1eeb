// kernels_packed.cuh -- two pointing windows per 2D FFT.
//
// The windows A I' of two slots a and b are real, so one complex transform carries both:
// Z = DFT2(z_a + i z_b), and with M(k) = conj(Z(-k)) the two spectra separate as
//     DFT2(z_a) = (Z + M) / 2,      DFT2(z_b) = (Z - M) / (2 i).
// Backwards, only Re IDFT2(G) is needed on each window, and Re IDFT2(G) = IDFT2(H) with the
// Hermitian part H(k) = (G(k) + conj G(-k)) / 2, whose inverse is real; so
//     IDFT2(H_a + i H_b) = Re IDFT2(G_a) + i Re IDFT2(G_b).
// Both identities pair the column kx with its mirror -kx: a column CTA holds the columns
// c0 .. c0 + ncol - 1 of [0, nf/2) and their mirrors (nf - c) mod nf, with column 0 (its own
// mirror) replaced by column nf/2 (also its own mirror) in the mirror half. The row passes
// carry slot a in the real and slot b in the imaginary part. An odd last slot runs with an
// empty partner (zero input, nothing written).
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "kernels_nufft.cuh"

namespace ivis {

// wts[k][q][p] I'[q][p] of one slot (bilinear through the pointing's grid if it has one),
// zero off the sky; wts is the beam, or the beam times the deapodisation dinv[p] dinv[q]
// (precomputed per pointing at prepare).
template <typename T>
__device__ __forceinline__ T window_value(const PairInfo &pi, int q, int p, const T *__restrict__ sky,
                                          const T *__restrict__ wts, const float2 *__restrict__ grids,
                                          int n, int nb) {
    const T a = wts[((size_t)pi.k * nb + q) * nb + p];
    const T *img = sky + (size_t)pi.chan * n * n;
    if (pi.gridded) {
        const float2 g = grids[((size_t)pi.k * nb + q) * nb + p];
        return a * bilerp(img, n, g.x, g.y);
    }
    const int y = pi.cy - nb / 2 + q, x = pi.cx - nb / 2 + p;
    return (y >= 0 && y < n && x >= 0 && x < n) ? a * img[(size_t)y * n + x] : (T)0;
}

// Column held by line L of a packed column CTA (2 ncol lines), and the line holding its mirror.
__device__ __forceinline__ int pk_col(int L, int c0, int ncol, int nf) {
    if (L < ncol) return c0 + L;
    const int c = c0 + L - ncol;
    return c == 0 ? nf / 2 : nf - c;
}
__device__ __forceinline__ int pk_mirror_line(int L, int c0, int ncol) {
    if (L < ncol) return (c0 + L == 0) ? 0 : L + ncol;
    return (c0 + L - ncol == 0) ? L : L - ncol;
}

// ------------------------------------------------------------------------- forward rows
// Line l: window row q of the slot pair (2 blockIdx.y, 2 blockIdx.y + 1) -> DFT along x.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 4)
k_fwd_rows_pk(const T *__restrict__ sky, const T *__restrict__ wts, const PairInfo *__restrict__ pinfo,
              int nslot, typename cplx_of<T>::type *rowbuf, int n, int nb,
              int lognf, const typename cplx_of<T>::type *__restrict__ tw, const float2 *__restrict__ grids) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, tpl = nf >> 4, lpb = blockDim.x / tpl;
    const int sa = 2 * blockIdx.y, sb = sa + 1;
    const PairInfo pa = pinfo[sa];
    const bool hasb = sb < nslot;
    const PairInfo pb = hasb ? pinfo[sb] : pa;
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int q = blockIdx.x * lpb + l;
    // element e of the line holds window column p = e + nb/2 (mod nf) if p < nb, else zero: the
    // thread's elements j0 + m tpl (the inputs of its first-pass butterfly, which runs from
    // registers) hold the columns j0 + ((m + 4) mod 16) tpl, those with (m + 4) mod 16 < 8 inside
    C in[16];
    if (!pa.gridded && !(hasb && pb.gridded)) {
        // windows on the sky grid (no re-projection): every gather is a predicated load with
        // no branch between them, so all of the thread's loads can be in flight at once
        const int qq = q < nb ? q : 0;
        const int ya = pa.cy - nb / 2 + qq, yb = pb.cy - nb / 2 + qq;
        const bool ra = q < nb && ya >= 0 && ya < n, rb = hasb && q < nb && yb >= 0 && yb < n;
        const T *wa = wts + ((size_t)pa.k * nb + qq) * nb, *wb = wts + ((size_t)pb.k * nb + qq) * nb;
        const T *ia = sky + (size_t)pa.chan * n * n + (size_t)(ra ? ya : 0) * n;
        const T *ib = sky + (size_t)pb.chan * n * n + (size_t)(rb ? yb : 0) * n;
        const int xa0 = pa.cx - nb / 2, xb0 = pb.cx - nb / 2;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int mp = (m + 4) & 15, p = j0 + mp * tpl;
            T va = (T)0, vb = (T)0;
            if (mp < 8) {
                const int xa = xa0 + p, xb = xb0 + p;
                if (ra && xa >= 0 && xa < n) va = wa[p] * ia[xa];
                if (rb && xb >= 0 && xb < n) vb = wb[p] * ib[xb];
            }
            in[m] = mk(va, vb);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int mp = (m + 4) & 15, p = j0 + mp * tpl;
            C v = mk((T)0, (T)0);
            if (mp < 8 && q < nb) {
                const T va = window_value(pa, q, p, sky, wts, grids, n, nb);
                const T vb = hasb ? window_value(pb, q, p, sky, wts, grids, n, nb) : (T)0;
                v = mk(va, vb);
            }
            in[m] = v;
        }
    }
    first_pass_regs<C, -1>(s, 1, l * nf, j0, in);
    __syncthreads();
    line_fft_from<C, -1>(s, 1, l * nf, lognf, j0, tw, 4, true);
    if (q < nb) {  // the last pass's elements j0 + m tpl straight to the packed row buffer
        C *out = rowbuf + ((size_t)blockIdx.y * nb + q) * nf;
        last_pass_regs<C, -1>(s, 1, l * nf, lognf, j0, tw, [&](int m, const C &v) { out[j0 + m * tpl] = v; });
    }
}

// ---------------------------------------------------------------------- forward columns
// DFT along y of the packed rows, then the two spectra to F[slot a] and F[slot b] (rows
// 0 .. nf/2; the rest follows from Hermitian symmetry).
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_fwd_cols_pk(const typename cplx_of<T>::type *__restrict__ rowbuf, typename cplx_of<T>::type *F,
              int nslot, int nb, int lognf, int logc, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, ncol = 1 << logc, nl = 2 * ncol, lgl = logc + 1, tpl = nf >> 4;
    const int c0 = blockIdx.x * ncol, pk = blockIdx.y;
    const int L = threadIdx.x & (nl - 1), j0 = threadIdx.x >> lgl;
    const int col = pk_col(L, c0, ncol, nf);
    const C *src = rowbuf + (size_t)pk * nb * nf;
    // nb = nf / 2 rows: 8 per thread (rows j0 + r tpl). Element e of the line holds row
    // (e + nb/2) mod nf (zero past nb), so element j0 + m tpl holds row j0 + ((m + 4) mod 16) tpl:
    // the thread's rows are the inputs of its own first-pass butterfly, which runs from registers
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = src[(size_t)(j0 + r * tpl) * nf + col];
    C in[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) in[m] = ((m + 4) & 15) < 8 ? v[(m + 4) & 15] : mk((T)0, (T)0);
    first_pass_regs<C, -1>(s, nl, L, j0, in);
    __syncthreads();
    line_fft_from<C, -1>(s, nl, L, lognf, j0, tw, 4, false);
    const int Lm = pk_mirror_line(L, c0, ncol);
    const int sa = 2 * pk, sb = sa + 1;
    C *Fa = F + (size_t)sa * nf * nf, *Fb = F + (size_t)sb * nf * nf;
    const bool hasb = sb < nslot;
    // each window is real, so its spectrum is Hermitian, F(-k) = conj F(k): only the rows
    // 0 .. nf/2 are written; the gridding passes read the other half mirrored
    for (int e = j0; e <= nf / 2; e += tpl) {
        const C z = s[pidx((e << lgl) + L)];
        const C zm = s[pidx((((nf - e) & (nf - 1)) << lgl) + Lm)];  // Z(-ky, -kx)
        Fa[(size_t)e * nf + col] = mk((T)0.5 * (z.x + zm.x), (T)0.5 * (z.y - zm.y));
        if (hasb) Fb[(size_t)e * nf + col] = mk((T)0.5 * (z.y + zm.y), (T)0.5 * (zm.x - z.x));
    }
}

// ---------------------------------------------------------------------- adjoint columns
// Z = H_a + i H_b from the two adjoint grids, inverse DFT along y, the nb window rows to the
// packed row buffer. The grids arrive folded onto rows 0 .. nf/2 (the rows past nf/2 are zero
// and stay so): only those rows are read; k_clear_half clears them afterwards.
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_adj_cols_pk(typename cplx_of<T>::type *G, typename cplx_of<T>::type *rowbuf, int nslot, int nb,
              int lognf, int logc, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, ncol = 1 << logc, nl = 2 * ncol, lgl = logc + 1, tpl = nf >> 4;
    const int c0 = blockIdx.x * ncol, pk = blockIdx.y;
    const int L = threadIdx.x & (nl - 1), j0 = threadIdx.x >> lgl;
    const int col = pk_col(L, c0, ncol, nf), colm = pk_col(pk_mirror_line(L, c0, ncol), c0, ncol, nf);
    const int sa = 2 * pk, sb = sa + 1;
    const bool hasb = sb < nslot;
    C *Ga = G + (size_t)sa * nf * nf, *Gb = G + (size_t)sb * nf * nf;
    // 16 rows e = j0 + k tpl per thread. The gridding pass folded the rows past nf/2 onto their
    // mirrors, so a row below nf/2 (k < 8) has only its own cells (a, b) and a row past it
    // (k >= 8) only its mirrors' (am, bm); rows 0 and nf/2 (k = 0 and 8 of thread j0 = 0) have
    // both. Four rows are loaded at a time (8 loads in flight), into the first-pass inputs.
    const C z0 = mk((T)0, (T)0);
    C in[16];  // element j0 + k tpl of the line, k = 4h + r: the inputs of this thread's first-pass butterfly
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const bool own = h < 2;  // rows k < 8 hold their own cells, rows k >= 8 their mirrors'
        C x[4], y[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = j0 + (4 * h + r) * tpl;
            const size_t i = own ? (size_t)e * nf + col : (size_t)(nf - e) * nf + colm;
            x[r] = Ga[i];
            y[r] = hasb ? Gb[i] : z0;
        }
        C xe = z0, ye = z0;  // row 0's mirror cell (h = 0) or row nf/2's own cell (h = 2)
        if (j0 == 0 && (h & 1) == 0) {
            const size_t i = own ? (size_t)colm : (size_t)(nf / 2) * nf + col;
            xe = Ga[i];
            ye = hasb ? Gb[i] : z0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const bool edge = r == 0 && j0 == 0 && (h & 1) == 0;
            const C a = own ? x[r] : (edge ? xe : z0), am = own ? (edge ? xe : z0) : x[r];
            const C b = own ? y[r] : (edge ? ye : z0), bm = own ? (edge ? ye : z0) : y[r];
            // H_a = (a + conj am)/2, H_b = (b + conj bm)/2, Z = H_a + i H_b
            const C ha = mk((T)0.5 * (a.x + am.x), (T)0.5 * (a.y - am.y));
            const C hb = mk((T)0.5 * (b.x + bm.x), (T)0.5 * (b.y - bm.y));
            in[4 * h + r] = mk(ha.x - hb.y, ha.y + hb.x);
        }
    }
    first_pass_regs<C, +1>(s, nl, L, j0, in);
    __syncthreads();
    line_fft_from<C, +1>(s, nl, L, lognf, j0, tw, 4, true);
    // element j0 + m tpl is window row j0 + ((m + 4) mod 16) tpl (row q at (q - nb/2) mod nf);
    // the rows q < nb go to the packed row buffer straight from registers
    C *dst = rowbuf + (size_t)pk * nb * nf;
    last_pass_regs<C, +1>(s, nl, L, lognf, j0, tw, [&](int m, const C &v) {
        const int mq = (m + 4) & 15;
        if (mq < 8) dst[(size_t)(j0 + mq * tpl) * nf + col] = v;
    });
}

// Rows 0 .. nf/2 of each of nslot adjoint grids back to zero for the next gridding pass: one
// contiguous run of (nf/2 + 1) nf cells per grid, cleared with 16-byte stores (whole cache
// lines, unlike zero stores from the column pass, which would cover 64-byte column segments).
// Grid: (CTAs per grid, nslot).
template <typename T>
__global__ void __launch_bounds__(256)
k_clear_half(typename cplx_of<T>::type *G, int lognf) {
    const int nf = 1 << lognf;
    // 16-byte stores per grid: rows 0 .. nf/2, (nf/2 + 1) nf cells of 8 (FP32) or 16 (FP64) bytes
    const int run = (int)((size_t)(nf / 2 + 1) * nf * sizeof(typename cplx_of<T>::type) / 16);
    float4 *g = reinterpret_cast<float4 *>(G + (size_t)blockIdx.y * nf * nf);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < run; i += gridDim.x * blockDim.x)
        g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------------- adjoint rows
// Inverse DFT along x; the real part is slot a's window gradient, the imaginary part slot b's.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 4)
k_adj_rows_pk(const typename cplx_of<T>::type *__restrict__ rowbuf, const T *__restrict__ wts,
              const PairInfo *__restrict__ pinfo, int nslot, T *contrib, int n,
              int nb, int lognf, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, tpl = nf >> 4, lpb = blockDim.x / tpl;
    const int sa = 2 * blockIdx.y, sb = sa + 1;
    const bool hasb = sb < nslot;
    const PairInfo pa = pinfo[sa];
    const PairInfo pb = hasb ? pinfo[sb] : pa;
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int q = blockIdx.x * lpb + l;
    {   // elements j0 + k tpl: the inputs of this thread's first-pass butterfly, from registers
        C in[16];
        const C *src = rowbuf + ((size_t)blockIdx.y * nb + (q < nb ? q : 0)) * nf;
#pragma unroll
        for (int k = 0; k < 16; ++k) in[k] = q < nb ? src[j0 + k * tpl] : mk((T)0, (T)0);
        first_pass_regs<C, +1>(s, 1, l * nf, j0, in);
    }
    __syncthreads();
    line_fft_from<C, +1>(s, 1, l * nf, lognf, j0, tw, 4, true);
    if (q >= nb) return;  // the line's last pass only feeds this row's outputs
    const int ya = pa.cy - nb / 2 + q, yb = pb.cy - nb / 2 + q;
    const bool ona = pa.gridded || (ya >= 0 && ya < n), onb = hasb && (pb.gridded || (yb >= 0 && yb < n));
    T *oa = contrib + ((size_t)sa * nb + q) * nb, *ob = contrib + ((size_t)sb * nb + q) * nb;
    const T *ba = wts + ((size_t)pa.k * nb + q) * nb, *bb = wts + ((size_t)pb.k * nb + q) * nb;
    // element j0 + m tpl is window column j0 + ((m + 4) mod 16) tpl (column p at (p - nb/2) mod
    // nf); the columns p < nb straight from registers
    last_pass_regs<C, +1>(s, 1, l * nf, lognf, j0, tw, [&](int m, const C &v) {
        const int mp = (m + 4) & 15, p = j0 + mp * tpl;
        if (mp >= 8) return;
        if (ona) oa[p] = v.x * ba[p];
        if (onb) ob[p] = v.y * bb[p];
    });
}

// ---------------------------------------------------------------- Toeplitz, packed pairs
// Column DFT of the packed rows, separation, products with the two spectra recombined as
// W = That_a Z_a + i That_b Z_b, inverse column DFT, the nb window rows back (in place).
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_toep_cols_pk(typename cplx_of<T>::type *rowbuf, const T *const *__restrict__ that_ptr, int nslot, int nb,
               int lognf, int logc, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, ncol = 1 << logc, nl = 2 * ncol, lgl = logc + 1, tpl = nf >> 4;
    const int c0 = blockIdx.x * ncol, pk = blockIdx.y;
    const int L = threadIdx.x & (nl - 1), j0 = threadIdx.x >> lgl;
    const int col = pk_col(L, c0, ncol, nf), Lm = pk_mirror_line(L, c0, ncol);
    const int sa = 2 * pk, sb = sa + 1;
    const bool hasb = sb < nslot;
    for (int e = j0; e < nf; e += tpl) s[pidx((e << lgl) + L)] = mk((T)0, (T)0);
    __syncthreads();
    C *buf = rowbuf + (size_t)pk * nb * nf;
    for (int q = j0; q < nb; q += tpl) s[pidx((((q - nb / 2) & (nf - 1)) << lgl) + L)] = buf[(size_t)q * nf + col];
    __syncthreads();
    line_fft<C, -1>(s, nl, L, lognf, j0, tw);
    const T *tha = that_ptr[sa] + (size_t)col * nf;
    const T *thb = hasb ? that_ptr[sb] + (size_t)col * nf : tha;
    C w[16];  // nf / tpl = 16 elements per thread
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = j0 + i * tpl;
        const C z = s[pidx((e << lgl) + L)];
        const C zm = s[pidx((((nf - e) & (nf - 1)) << lgl) + Lm)];
        const C za = mk((T)0.5 * (z.x + zm.x), (T)0.5 * (z.y - zm.y));
        const C zb = mk((T)0.5 * (z.y + zm.y), (T)0.5 * (zm.x - z.x));
        const T ta = tha[e], tb = hasb ? thb[e] : (T)0;
        w[i] = mk(ta * za.x - tb * zb.y, ta * za.y + tb * zb.x);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) s[pidx(((j0 + i * tpl) << lgl) + L)] = w[i];
    __syncthreads();
    line_fft_from<C, +1>(s, nl, L, lognf, j0, tw, 0, true);
    // the window rows q < nb (element j0 + m tpl is row j0 + ((m + 4) mod 16) tpl) from registers
    last_pass_regs<C, +1>(s, nl, L, lognf, j0, tw, [&](int m, const C &v) {
        const int mq = (m + 4) & 15;
        if (mq < 8) buf[(size_t)(j0 + mq * tpl) * nf + col] = v;
    });
}

// Row pass of the packed Toeplitz form: y_a = Re, y_b = Im of the inverse row DFT; per slot
// the gradient times the beam and the cost partial z (y/2 - b) (+ C in the first CTA).
template <typename T>
__global__ void __launch_bounds__(256)
k_toep_rows_pk(const typename cplx_of<T>::type *__restrict__ rowbuf, const T *__restrict__ sky,
               const T *__restrict__ beams, const PairInfo *__restrict__ pinfo, int nslot,
               const T *const *__restrict__ bwin_ptr, const double *__restrict__ qconst, T *contrib,
               double *jpart, int n, int nb, int lognf, const typename cplx_of<T>::type *__restrict__ tw,
               const float2 *__restrict__ grids) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    __shared__ double red[32];
    const int nf = 1 << lognf, tpl = nf >> 4, lpb = blockDim.x / tpl;
    const int sa = 2 * blockIdx.y, sb = sa + 1;
    const bool hasb = sb < nslot;
    const PairInfo pa = pinfo[sa];
    const PairInfo pb = hasb ? pinfo[sb] : pa;
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int q = blockIdx.x * lpb + l;
    if (q < nb) {
        const C *src = rowbuf + ((size_t)blockIdx.y * nb + q) * nf;
        for (int e = j0; e < nf; e += tpl) s[pidx(l * nf + e)] = src[e];
    }
    __syncthreads();
    line_fft_from<C, +1>(s, 1, l * nf, lognf, j0, tw, 0, true);
    T acc_a = (T)0, acc_b = (T)0;  // nb / tpl terms per thread in the working precision
    if (q < nb) {
        const int ya = pa.cy - nb / 2 + q, yb = pb.cy - nb / 2 + q;
        const bool ona = pa.gridded || (ya >= 0 && ya < n), onb = hasb && (pb.gridded || (yb >= 0 && yb < n));
        T *oa = contrib + ((size_t)sa * nb + q) * nb, *ob = contrib + ((size_t)sb * nb + q) * nb;
        const T *ba = beams + ((size_t)pa.k * nb + q) * nb, *bb = beams + ((size_t)pb.k * nb + q) * nb;
        const T *wa = bwin_ptr[sa] + (size_t)q * nb, *wb = hasb ? bwin_ptr[sb] + (size_t)q * nb : wa;
        // the last pass in registers: element j0 + m tpl is window column j0 + ((m + 4) mod 16) tpl
        last_pass_regs<C, +1>(s, 1, l * nf, lognf, j0, tw, [&](int m, const C &v) {
            const int mp = (m + 4) & 15, p = j0 + mp * tpl;
            if (mp >= 8) return;
            if (ona) {
                const T z = window_value(pa, q, p, sky, beams, grids, n, nb);
                oa[p] = ba[p] * (v.x - wa[p]);
                acc_a += z * (v.x * (T)0.5 - wa[p]);
            }
            if (onb) {
                const T z = window_value(pb, q, p, sky, beams, grids, n, nb);
                ob[p] = bb[p] * (v.y - wb[p]);
                acc_b += z * (v.y * (T)0.5 - wb[p]);
            }
        });
    }
    const double sa_ = block_sum_t(acc_a, red);
    if (threadIdx.x == 0) jpart[(size_t)sa * gridDim.x + blockIdx.x] = sa_ + (blockIdx.x == 0 ? qconst[sa] : 0.0);
    __syncthreads();
    const double sb_ = block_sum_t(acc_b, red);
    if (hasb && threadIdx.x == 0) jpart[(size_t)sb * gridDim.x + blockIdx.x] = sb_ + (blockIdx.x == 0 ? qconst[sb] : 0.0);
}

}  // namespace ivis
