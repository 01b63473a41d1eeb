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

// One CTA per TE x TE pixel tile of one channel (256 threads; TE = 32: 4 pixels each, TE = 16
// for small images so that the grid still fills the GPU: 1 pixel each). The Laplacian
// terms come from the tile's sky with a 2-pixel halo and its Laplacian with a 1-pixel halo,
// both staged in shared memory; the window contributions from the channel's pairs whose windows
// meet the tile, listed once per CTA in the channel's slot order (the per-pixel sum runs in
// that order, as it would over all the channel's pairs). One R partial per CTA.
template <typename T, int TE>
__global__ void __launch_bounds__(256)
k_assemble(const T *__restrict__ sky, const T *__restrict__ contrib,
           const PairInfo *__restrict__ pinfo, const int *__restrict__ chan_start,
           const int *__restrict__ chan_list, const T *__restrict__ gradK, T *grad, int n, int nb,
           int nchan, T lr, T ls, int use_r, int use_k, double *rpart) {
    constexpr int PPT = TE * TE / 256, RSTEP = 256 / TE;  // pixels per thread, rows per pass
    __shared__ T xs[TE + 4][TE + 5];  // sky, 2-pixel halo, zero off the image
    __shared__ T lp[TE + 2][TE + 3];  // Laplacian, 1-pixel halo
    __shared__ int list[256];
    __shared__ int nlist;
    __shared__ double red[32];
    (void)nchan;
    const int ntx = (n + TE - 1) / TE;
    const int chan = blockIdx.y;
    const int y0 = (blockIdx.x / ntx) * TE, x0 = (blockIdx.x % ntx) * TE;
    const int tx = threadIdx.x % TE, ty = threadIdx.x / TE;  // pixel (y0 + ty + RSTEP j, x0 + tx)
    const size_t npix = (size_t)n * n;
    const T *I = sky + (size_t)chan * npix;
    if (use_r) {
        for (int i = threadIdx.x; i < (TE + 4) * (TE + 4); i += blockDim.x) {
            const int yy = i / (TE + 4), xx = i - yy * (TE + 4);
            xs[yy][xx] = pix(I, n, y0 - 2 + yy, x0 - 2 + xx);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < (TE + 2) * (TE + 2); i += blockDim.x) {
            const int yy = i / (TE + 2), xx = i - yy * (TE + 2);
            lp[yy][xx] = (T)4 * xs[yy + 1][xx + 1] - xs[yy][xx + 1] - xs[yy + 2][xx + 1] - xs[yy + 1][xx] -
                         xs[yy + 1][xx + 2];
        }
    }
    T g[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) g[j] = (T)0;
    const int t0 = chan_start[chan], t1 = chan_start[chan + 1];
    for (int b0 = t0; b0 < t1; b0 += 256) {
        const int b1 = min(t1, b0 + 256);
        __syncthreads();  // the previous batch's list is read
        if (threadIdx.x < 32) {  // warp 0 lists the batch's windows that meet the tile, in order
            int cnt = 0;
            for (int c0 = b0; c0 < b1; c0 += 32) {
                const int t = c0 + threadIdx.x;
                bool cov = false;
                int slot = 0;
                if (t < b1) {
                    slot = chan_list[t];
                    const PairInfo pi = pinfo[slot];
                    const int wy = pi.cy - nb / 2, wx = pi.cx - nb / 2;
                    // pointings with a re-projection grid are added by k_grid_scatter
                    cov = !pi.gridded && wy < y0 + TE && wy + nb > y0 && wx < x0 + TE && wx + nb > x0;
                }
                const unsigned m = __ballot_sync(0xffffffffu, cov);
                if (cov) list[cnt + __popc(m & ((1u << threadIdx.x) - 1u))] = slot;
                cnt += __popc(m);
            }
            if (threadIdx.x == 0) nlist = cnt;
        }
        __syncthreads();
        for (int k = 0; k < nlist; ++k) {
            const int slot = list[k];
            const PairInfo pi = pinfo[slot];
            const int p = x0 + tx - (pi.cx - nb / 2);
            const T *cs = contrib + (size_t)slot * nb * nb;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int q = y0 + ty + RSTEP * j - (pi.cy - nb / 2);
                if ((unsigned)q < (unsigned)nb && (unsigned)p < (unsigned)nb) g[j] += cs[(size_t)q * nb + p];
            }
        }
    }
    __syncthreads();  // the Laplacian tile is complete
    T rloc = (T)0;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int ly = ty + RSTEP * j, y = y0 + ly, x = x0 + tx;
        if (y >= n || x >= n) continue;
        const size_t idx = (size_t)chan * npix + (size_t)y * n + x;
        T gj = g[j];
        if (use_r) {
            const T d0 = lp[ly + 1][tx + 1];
            T gr = (T)4 * d0;
            if (y > 0) gr -= lp[ly][tx + 1];
            if (y < n - 1) gr -= lp[ly + 2][tx + 1];
            if (x > 0) gr -= lp[ly + 1][tx];
            if (x < n - 1) gr -= lp[ly + 1][tx + 2];
            gj += lr * gr;
            rloc += (T)0.5 * d0 * d0;
        }
        if (use_k) gj += ls * gradK[idx];
        grad[idx] = gj;
    }
    const double s = block_sum_t(rloc, red);
    if (threadIdx.x == 0) rpart[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Tile edge of k_assemble: 32, or 16 when 32-pixel tiles would give fewer than 1184 CTAs.
inline int assemble_te(int n, int nchan) {
    const long long nt = (n + 31) / 32;
    return nt * nt * nchan < 1184 ? 16 : 32;
}
// CTAs of k_assemble: (tiles per channel, channels).
inline dim3 assemble_grid(int n, int nchan) {
    const int te = assemble_te(n, nchan), nt = (n + te - 1) / te;
    return dim3((unsigned)(nt * nt), (unsigned)nchan);
}

// Separable dish-beam convolution, one axis per launch: out = sum_{t=-R..R} b_c[t] in(. - t),
// zero outside the image. A CTA covers 32 lines (one per lane) x CONV_TO outputs along the
// convolution axis. Warp w produces CONV_OPT consecutive outputs (w % CONV_NWO) over one of
// CONV_SPLIT segments of the taps (w / CONV_NWO) from a sliding window of registers, so each
// shared-memory load feeds CONV_OPT FMAs; the window is a ring indexed by the tap step modulo
// CONV_OPT (taps unrolled by CONV_OPT, no register moves); the segments are summed through
// shared memory in a fixed order. The staged strip is laid out [position][line] with a
// 33-word pitch (rows pass: lines are image rows and the transpose would otherwise serialise
// on one bank). 32-output strips keep the grid at >= 2 CTAs per SM on a 512^2 image.
constexpr int CONV_OPT = 8;
constexpr int CONV_NWO = 4;                            // output warps per tap segment
constexpr int CONV_TO = CONV_NWO * CONV_OPT;           // outputs per CTA along the axis
constexpr int CONV_SPLIT = 4;                          // tap segments
constexpr int CONV_THREADS = 32 * CONV_NWO * CONV_SPLIT;

// AXIS 0: along x (lines = rows); AXIS 1: along y (lines = columns).
// FUSED (AXIS 1 only): out = e = (t - T)/sigma^2 and the CTA's share of K goes to kpart.
template <typename T, int AXIS, int FUSED>
__global__ void __launch_bounds__(CONV_THREADS)
k_conv_axis(const T *__restrict__ in, T *out, const T *__restrict__ taps, int R, int n,
            const T *__restrict__ tsd, const double *__restrict__ inv_sig2, double *kpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const int P = 33;
    const int L = CONV_TO + 2 * R;  // staged positions
    constexpr int NPART = (CONV_SPLIT - 1) * CONV_NWO * CONV_OPT * 32;
    T *sh = reinterpret_cast<T *>(smem_raw);
    T *tp = sh + max(L * P, NPART);
    T *part = sh;  // [CONV_SPLIT - 1][CONV_NWO][CONV_OPT][32], reuses the strip after the taps loop
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wo = wid % CONV_NWO, seg = wid / CONV_NWO;
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
    const int o0 = wo * CONV_OPT;
    const int ntap = 2 * R + 1;
    const int tb = seg * ntap / CONV_SPLIT, te = (seg + 1) * ntap / CONV_SPLIT;
    T acc[CONV_OPT], win[CONV_OPT];
#pragma unroll
    for (int j = 0; j < CONV_OPT; ++j) {
        acc[j] = (T)0;
        win[j] = sh[(o0 + j + 2 * R - tb) * P + lane];
    }
    // at step u of a block of CONV_OPT taps, logical window entry j is win[(j - u) mod OPT];
    // the entry dropped after step u takes the next staged value
    int t = tb;
    for (; t + CONV_OPT <= te; t += CONV_OPT) {
#pragma unroll
        for (int u = 0; u < CONV_OPT; ++u) {
            const T bt = tp[t + u];
#pragma unroll
            for (int j = 0; j < CONV_OPT; ++j) acc[j] += bt * win[(j - u + CONV_OPT) % CONV_OPT];
            win[(CONV_OPT - 1 - u) % CONV_OPT] = sh[max(o0 + 2 * R - (t + u) - 1, 0) * P + lane];
        }
    }
    for (; t < te; ++t) {
        const T bt = tp[t];
#pragma unroll
        for (int j = 0; j < CONV_OPT; ++j) acc[j] += bt * win[j];
#pragma unroll
        for (int j = CONV_OPT - 1; j > 0; --j) win[j] = win[j - 1];
        win[0] = sh[max(o0 + 2 * R - t - 1, 0) * P + lane];
    }
    __syncthreads();  // every warp is done reading the strip
    if (seg > 0) {
#pragma unroll
        for (int j = 0; j < CONV_OPT; ++j) part[(((seg - 1) * CONV_NWO + wo) * CONV_OPT + j) * 32 + lane] = acc[j];
    }
    __syncthreads();
    T kloc = (T)0;  // <= CONV_OPT terms per thread in the working precision, then FP64
    if (seg == 0) {
#pragma unroll
        for (int q = 1; q < CONV_SPLIT; ++q)
#pragma unroll
            for (int j = 0; j < CONV_OPT; ++j) acc[j] += part[(((q - 1) * CONV_NWO + wo) * CONV_OPT + j) * 32 + lane];
        const T is2 = FUSED ? (T)inv_sig2[c] : (T)0;
        const int line = line0 + lane;
#pragma unroll
        for (int j = 0; j < CONV_OPT; ++j) {
            const int pos = pos0 + o0 + j;
            if (line >= n || pos >= n) continue;
            const size_t o = AXIS == 0 ? ((size_t)c * n + line) * n + pos : ((size_t)c * n + pos) * n + line;
            if (FUSED) {
                const T e = acc[j] - tsd[o];
                kloc += (T)0.5 * e * e * is2;
                out[o] = e * is2;
            } else {
                out[o] = acc[j];
            }
        }
    }
    if (FUSED) {
        const double sum = block_sum((double)kloc, red);
        if (threadIdx.x == 0)
            kpart[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum;
    }
}

// out[0..3] = {Q_tot, Q, K, R} from the FP64 partials. FP64 issue is scarce on this part (a
// few lanes per clock per SM), so the sums are spread over FIN_BLOCKS CTAs: each CTA adds its
// grid-strided share of the three partial arrays and writes three block sums to out[4..];
// the last CTA to finish (atomic ticket in the word after them, reset for the next call)
// adds the block sums in index order. Fixed summation order for a fixed launch shape.
constexpr int FIN_BLOCKS = 32;
constexpr int FIN_WORDS = 4 + 3 * FIN_BLOCKS + 1;  // doubles of the cost record incl. scratch

__global__ void __launch_bounds__(256)
k_finalize(const double *__restrict__ jpart, int nj, const double *__restrict__ kpart, int nk,
           const double *__restrict__ rpart, int nr, double lr, double ls, double *out) {
    __shared__ double red[3][32];
    __shared__ int last;
    double *bp = out + 4;
    unsigned *ticket = reinterpret_cast<unsigned *>(out + 4 + 3 * FIN_BLOCKS);
    const int G = gridDim.x * blockDim.x, gt = blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    for (int i = gt; i < nj; i += G) v[0] += __ldcg(jpart + i);
    for (int i = gt; i < nk; i += G) v[1] += __ldcg(kpart + i);
    for (int i = gt; i < nr; i += G) v[2] += __ldcg(rpart + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) red[a][wid] = v[a];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = lane < nw ? red[a][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) bp[3 * blockIdx.x + a] = v[a];
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last || wid != 0) return;
    __threadfence();
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = lane < (int)gridDim.x ? __ldcg(bp + 3 * lane + a) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
    if (lane == 0) {
        out[1] = v[0];
        out[2] = v[1];
        out[3] = v[2];
        out[0] = v[0] + ls * v[1] + lr * v[2];
        *ticket = 0u;
    }
}

// Beam-weight map b[y][x] = sum over pointings covering (y, x) of A_k[q][p]^2 (the weight of
// a linear mosaic, Sect. 4.3); used as an input plane of the learned warm start.
template <typename T>
__global__ void k_beam_weight(const T *__restrict__ beams, const int *__restrict__ cx,
                              const int *__restrict__ cy, const int *__restrict__ gridded,
                              int npoint, int n, int nb, T *out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    const int y = (int)(idx / n), x = (int)(idx % n);
    T s = (T)0;
    for (int k = 0; k < npoint; ++k) {
        if (gridded[k]) continue;
        const int q = y - (cy[k] - nb / 2), p = x - (cx[k] - nb / 2);
        if ((unsigned)q < (unsigned)nb && (unsigned)p < (unsigned)nb) {
            const T a = beams[((size_t)k * nb + q) * nb + p];
            s += a * a;
        }
    }
    out[idx] = s;
}

// Adjoint of the bilinear re-projection for gridded pointings: grad[chan] += B_k^T contrib_k.
// One thread per window pixel of every slot (non-gridded slots return at once).
template <typename T>
__global__ void k_grid_scatter(const T *__restrict__ contrib, const PairInfo *__restrict__ pinfo,
                               const float2 *__restrict__ grids, T *grad, int n, int nb) {
    const int slot = blockIdx.y;
    const PairInfo pi = pinfo[slot];
    if (!pi.gridded) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nb) return;
    const float2 g = grids[(size_t)pi.k * nb * nb + i];
    bilerp_adj(grad + (size_t)pi.chan * n * n, n, g.x, g.y, contrib[(size_t)slot * nb * nb + i]);
}

// Beam-weight map contribution of gridded pointings: out += B_k^T (A_k^2).
template <typename T>
__global__ void k_beam_weight_grid(const T *__restrict__ beams, const float2 *__restrict__ grids,
                                   const int *__restrict__ gridded, int n, int nb, T *out) {
    const int k = blockIdx.y;
    if (!gridded[k]) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nb) return;
    const T a = beams[(size_t)k * nb * nb + i];
    const float2 g = grids[(size_t)k * nb * nb + i];
    bilerp_adj(out, n, g.x, g.y, a * a);
}

// out[k][q][p] = beams[k][q][p] dinv[p] dinv[q] for every pointing (n = npoint nb^2).
template <typename T>
__global__ void k_beam_deapod(const T *__restrict__ beams, const T *__restrict__ dinv, int nb, size_t n,
                              T *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = (int)(i % nb), q = (int)((i / nb) % nb);
    out[i] = beams[i] * dinv[p] * dinv[q];
}

template <typename T>
__global__ void k_scale(size_t n, const T *__restrict__ in, T a, T *out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * in[i];
}

template <typename T>
__global__ void k_f32_to(const float *__restrict__ in, T *out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}

}  // namespace ivis
