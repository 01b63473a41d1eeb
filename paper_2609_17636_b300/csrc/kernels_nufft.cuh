// kernels_nufft.cuh -- the per-pointing NUFFT pair of the data term (paper Eqs. 3-6).
//
// Forward (type 2, image -> visibilities), for each (pointing, channel) pair:
//   a1  window gather x beam x deapodisation, zero-padded to the 2x oversampled grid,
//       fused into the row FFT                                         (k_fwd_rows)
//   a2  column FFT of the fine grid                                    (k_fwd_cols)
//   a3  interpolation with the ES kernel -> model visibilities, residual r = V~ - V,
//       J partial 1/2 w |r|^2 in FP64                                  (k_grid_pass)
// Adjoint (type 1, visibilities -> image), in the same pass and the reverse order:
//   a4  spreading of w r with the same kernel values into a shared-memory sub-grid,
//       flushed to the global adjoint grid with atomics                (k_grid_pass)
//   a5  column inverse FFT, keeping only the nb modes of the window    (k_adj_cols)
//       row inverse FFT + deapodisation + Re + beam                    (k_adj_rows)
//
// Conventions: fine grid nf = 2 nb; window mode k = p - nb/2 sits at grid index k mod nf;
// a visibility's grid coordinate is s = u * cell * nf (folded into [0, nf)); its W taps are
// cells g0 .. g0+W-1 with g0 = floor(s - W/2) + 1 and kernel argument (s - g)/(W/2).
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace ivis {

struct PairInfo {
    int k, chan, cx, cy;
    int gridded;  // 1: the window is the bilinear re-projection through the pointing's grid
    int wplane;   // 1: a w-plane slot of the full Eq. 1 (modulation by exp(-2 pi i wk x'))
    double wk;    // the plane's w (wavelengths)
};

// Bilinear interpolation of img (n x n, zero off the sky) at (X, Y) in pixel units (X along
// columns); non-finite or far-off coordinates give zero (Eq. 2, Sect. 3.3).
template <typename T>
__device__ __forceinline__ T bilerp(const T *__restrict__ img, int n, float X, float Y) {
    if (!(X > -2.0f && X < (float)n + 1.0f && Y > -2.0f && Y < (float)n + 1.0f)) return (T)0;
    const T xf = floor((T)X), yf = floor((T)Y);
    const int x0 = (int)xf, y0 = (int)yf;
    const T fx = (T)X - xf, fy = (T)Y - yf;
    T s = (T)0;
    if (y0 >= 0 && y0 < n) {
        if (x0 >= 0 && x0 < n) s += ((T)1 - fx) * ((T)1 - fy) * img[(size_t)y0 * n + x0];
        if (x0 + 1 >= 0 && x0 + 1 < n) s += fx * ((T)1 - fy) * img[(size_t)y0 * n + x0 + 1];
    }
    if (y0 + 1 >= 0 && y0 + 1 < n) {
        if (x0 >= 0 && x0 < n) s += ((T)1 - fx) * fy * img[(size_t)(y0 + 1) * n + x0];
        if (x0 + 1 >= 0 && x0 + 1 < n) s += fx * fy * img[(size_t)(y0 + 1) * n + x0 + 1];
    }
    return s;
}

// Transpose of bilerp: out += v spread with the same four weights (atomics).
template <typename T>
__device__ __forceinline__ void bilerp_adj(T *out, int n, float X, float Y, T v) {
    if (!(X > -2.0f && X < (float)n + 1.0f && Y > -2.0f && Y < (float)n + 1.0f)) return;
    const T xf = floor((T)X), yf = floor((T)Y);
    const int x0 = (int)xf, y0 = (int)yf;
    const T fx = (T)X - xf, fy = (T)Y - yf;
    if (y0 >= 0 && y0 < n) {
        if (x0 >= 0 && x0 < n) atomicAdd(&out[(size_t)y0 * n + x0], ((T)1 - fx) * ((T)1 - fy) * v);
        if (x0 + 1 >= 0 && x0 + 1 < n) atomicAdd(&out[(size_t)y0 * n + x0 + 1], fx * ((T)1 - fy) * v);
    }
    if (y0 + 1 >= 0 && y0 + 1 < n) {
        if (x0 >= 0 && x0 < n) atomicAdd(&out[(size_t)(y0 + 1) * n + x0], ((T)1 - fx) * fy * v);
        if (x0 + 1 >= 0 && x0 + 1 < n) atomicAdd(&out[(size_t)(y0 + 1) * n + x0 + 1], fx * fy * v);
    }
}

struct Chunk {
    int slot;    // active pair slot
    int tile;    // tile id within the pair's fine grid (ty * ntx + tx, ntx = nf / tile edge)
    int begin;   // first visibility (pair-local sorted index)
    int end;     // one past the last
};

template <typename T> struct coord_of;
template <> struct coord_of<float> { typedef uint2 type; };     // 12-bit cell | 20-bit fraction
template <> struct coord_of<double> { typedef double2 type; };  // folded grid coordinate

template <typename T> struct PairData {
    const typename coord_of<T>::type *coord;
    const typename cplx_of<T>::type *vis;
    const T *w;
    const int *orig;
    int m;
    long long pred_off;  // MODE_PREDICT writes pred[pred_off + orig[v]]
};

constexpr int FRAC_BITS = 20;
constexpr unsigned FRAC_ONE = 1u << FRAC_BITS;
constexpr int GTILE = 32;    // fine-grid bin edge (cells) of the visibility sort

// Order of the 32 x 32-cell bins in the sort: bins are grouped in 2 x 2 quads (row-major over
// the quads, then row-major inside a quad), so that both a 32-cell tile and a 64-cell tile own
// one contiguous run of the sorted visibilities. ntx = nf / 32 bins per row (a power of two).
__host__ __device__ __forceinline__ int bin_of_tile(int tx, int ty, int ntx) {
    if (ntx < 2) return ty * ntx + tx;
    const int h = ntx >> 1;
    return ((((ty >> 1) * h + (tx >> 1)) << 2) | ((ty & 1) << 1) | (tx & 1));
}
__host__ __device__ __forceinline__ void tile_of_bin(int j, int ntx, int &tx, int &ty) {
    if (ntx < 2) { tx = 0; ty = 0; return; }
    const int h = ntx >> 1, q = j >> 2, s = j & 3;
    tx = 2 * (q % h) + (s & 1);
    ty = 2 * (q / h) + (s >> 1);
}
constexpr int ES_MAXDEG = 18; // max degree of the per-tap kernel polynomials
// Degree W + 1: for W = 7 the interpolation error is 5.8e-8 (degree W + 2: 5.4e-8; the kernel's
// square-root edge sets the floor), far below the FP32 NUFFT's 1e-6.
template <int W> struct es_deg { static constexpr int value = W + 1 < ES_MAXDEG ? W + 1 : ES_MAXDEG; };

// Per-tap polynomials of the ES kernel (FP32 path): the x kernel value of tap t of a
// visibility whose first-tap fraction is f in [0, 1) is sum_i c[t][i] (2f - 1)^i. Fitted at
// plan time in FP64 by interpolation at Chebyshev nodes (see es_fit in ivis.cu).
template <int W>
__device__ __forceinline__ float es_poly(const float (&c)[es_deg<W>::value + 1], float f) {
    const float x = 2.0f * f - 1.0f;
    float acc = c[es_deg<W>::value];
#pragma unroll
    for (int i = es_deg<W>::value - 1; i >= 0; --i) acc = fmaf(acc, x, c[i]);
    return acc;
}

// ---------------------------------------------------------------- set-up: coordinates, sort
// Grid coordinate, tile key and validity of each input visibility.
template <typename T>
__global__ void k_vis_prepare(int m, const float *__restrict__ uvw, const float *__restrict__ vis,
                              const float *__restrict__ wt, double scale, int lognf, int W,
                              int tile, int ntx, typename coord_of<T>::type *coord_tmp,
                              int *key, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int nf = 1 << lognf;
    float u = uvw[3 * (size_t)i], v = uvw[3 * (size_t)i + 1];
    float vr = vis[2 * (size_t)i], vi = vis[2 * (size_t)i + 1], w = wt[i];
    if (!isfinite(u) || !isfinite(v) || !isfinite(vr) || !isfinite(vi) || !isfinite(w) || w < 0.f)
        atomicOr(err, 1);
    double sc[2] = {(double)u * scale, (double)v * scale};
    int g0[2];
    double half = 0.5 * W;
    unsigned packed[2];
    for (int a = 0; a < 2; ++a) {
        double s = sc[a] - nf * floor(sc[a] / nf);
        if (s >= nf) s -= nf;
        if (!(s >= 0.0)) s = 0.0;  // non-finite input: flagged above
        sc[a] = s;
        double gd = floor(s - half) + 1.0;
        long long g = (long long)gd;
        double frac = s - gd - (half - 1.0);
        unsigned q = (unsigned)(frac * (double)FRAC_ONE + 0.5);
        if (q >= FRAC_ONE) { q = 0; g += 1; }
        g = ((g % nf) + nf) % nf;
        if (sizeof(T) == 8) {  // the FP64 kernels recompute g0 from s: use the same rule
            long long g2 = (long long)(floor(s - half) + 1.0);
            g = ((g2 % nf) + nf) % nf;
        }
        g0[a] = (int)g;
        packed[a] = ((unsigned)g << FRAC_BITS) | q;
    }
    if constexpr (sizeof(T) == 4) {
        coord_tmp[i] = make_uint2(packed[0], packed[1]);
    } else {
        coord_tmp[i] = make_double2(sc[0], sc[1]);
    }
    // bin-major (bins in quad order), then the 8 x 8-cell block within the bin (row-major), then
    // the first-tap cell within the block (row-major): every bin and every block owns one
    // contiguous run of the sorted visibilities, and visibilities that share a first-tap cell
    // are adjacent
    const int cx = g0[0] % tile, cy = g0[1] % tile;
    key[i] = bin_of_tile(g0[0] / tile, g0[1] / tile, ntx) * tile * tile +
             ((cy >> 3) * (tile >> 3) + (cx >> 3)) * 64 + (cy & 7) * 8 + (cx & 7);
}

__global__ void k_hist(int m, const int *__restrict__ key, int *count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) atomicAdd(&count[key[i]], 1);
}

// Exclusive prefix sum of n ints (set-up only): per-1024 block scans, a scan of the block
// totals, then the block offsets added back.
__global__ void k_scan_block(int n, const int *__restrict__ in, int *out, int *bsum) {
    __shared__ int wsum[8];
    const int base = blockIdx.x * 1024 + threadIdx.x * 4;
    int v[4], t = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        t += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = t;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < wid; ++w) woff += wsum[w];
    int run = woff + incl - t;
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 255) bsum[blockIdx.x] = woff + incl;
}

// In-place exclusive scan of nb block totals by one CTA of 1024 threads.
__global__ void k_scan_top(int nb, int *bsum) {
    __shared__ int tmp[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        tmp[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int y = threadIdx.x >= o ? tmp[threadIdx.x - o] : 0;
            __syncthreads();
            tmp[threadIdx.x] += y;
            __syncthreads();
        }
        const int excl = tmp[threadIdx.x] - v + carry;
        __syncthreads();
        if (i < nb) bsum[i] = excl;
        if (threadIdx.x == 1023) carry += tmp[1023];
        __syncthreads();
    }
}

__global__ void k_scan_add(int n, int *out, const int *__restrict__ bsum) {
    const int i = blockIdx.x * 1024 + threadIdx.x * 4;
    const int off = bsum[blockIdx.x];
    for (int k = 0; k < 4; ++k)
        if (i + k < n) out[i + k] += off;
}

// start[t] = first sorted slot of bin t in sort order (t <= ntiles; start[ntiles] = m).
__global__ void k_tile_starts(int ntiles, int per_tile, int m, const int *__restrict__ cell_start,
                              int *start) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) start[t] = cell_start[(size_t)t * per_tile];
    if (t == ntiles) start[t] = m;
}

// Scatter into key order. cursor[key] starts at the key's first slot.
template <typename T>
__global__ void k_vis_scatter(int m, const int *__restrict__ key,
                              const typename coord_of<T>::type *__restrict__ coord_tmp,
                              const float *__restrict__ vis, const float *__restrict__ wt,
                              int *cursor, typename coord_of<T>::type *coord,
                              typename cplx_of<T>::type *vout, T *wout, int *orig) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int pos = atomicAdd(&cursor[key[i]], 1);
    coord[pos] = coord_tmp[i];
    vout[pos] = mk((T)vis[2 * (size_t)i], (T)vis[2 * (size_t)i + 1]);
    wout[pos] = (T)wt[i];
    orig[pos] = i;
}

// ------------------------------------------------------------------ forward row pass (a1)
// CTA = lpb window rows of one pair (tpl = nf/16 threads per row). blockIdx.x = row block.
template <typename T>
__global__ void __launch_bounds__(256)
k_fwd_rows(const T *__restrict__ sky, const T *__restrict__ beams,
           const PairInfo *__restrict__ pinfo, const T *__restrict__ dinv,
           typename cplx_of<T>::type *rowbuf, int n, int nb, int lognf,
           const typename cplx_of<T>::type *__restrict__ tw, const float2 *__restrict__ grids,
           const T *__restrict__ wx, const T *__restrict__ wcorr) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, tpl = nf >> 4, lpb = blockDim.x / tpl;
    const int slot = blockIdx.y;
    const PairInfo pi = pinfo[slot];
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int q = blockIdx.x * lpb + l;
    const int y = pi.cy - nb / 2 + q;
    const bool on = q < nb && (pi.gridded || (y >= 0 && y < n));
    // w-plane slot: window value times corr exp(-2 pi i wk x') (complex)
    auto put = [&](int p, T val) {
        C v = mk(val, (T)0);
        if (pi.wplane) {
            const size_t t = (size_t)q * nb + p;
            T sn, cs;
            sincospi_t((T)(-2.0 * pi.wk) * wx[t], &sn, &cs);
            const T a = val * wcorr[t];
            v = mk(a * cs, a * sn);
        }
        s[pidx(l * nf + ((p - nb / 2) & (nf - 1)))] = v;
    };
    C *line = s;  // element e of line l at s[pidx(l * nf + e)]
    for (int e = j0; e < nf; e += tpl) line[pidx(l * nf + e)] = mk((T)0, (T)0);
    __syncthreads();
    if (on) {
        const T *brow = beams + ((size_t)pi.k * nb + q) * nb;
        const T dq = dinv[q];
        if (pi.gridded) {
            const T *img = sky + (size_t)pi.chan * n * n;
            const float2 *grow = grids + ((size_t)pi.k * nb + q) * nb;
            for (int p = j0; p < nb; p += tpl) {
                const float2 g = grow[p];
                put(p, bilerp(img, n, g.x, g.y) * brow[p] * dinv[p] * dq);
            }
        } else {
            const T *srow = sky + ((size_t)pi.chan * n + y) * n;
            const int x0 = pi.cx - nb / 2;
            for (int p = j0; p < nb; p += tpl) {
                const int x = x0 + p;
                put(p, (x >= 0 && x < n) ? srow[x] * brow[p] * dinv[p] * dq : (T)0);
            }
        }
    }
    __syncthreads();
    line_fft<C, -1>(s, 1, l * nf, lognf, j0, tw);
    if (q < nb) {
        C *out = rowbuf + ((size_t)slot * nb + q) * nf;
        for (int e = j0; e < nf; e += tpl) out[e] = on ? line[pidx(l * nf + e)] : mk((T)0, (T)0);
    }
}

// ---------------------------------------------------------------- forward column pass (a2)
// CTA = ncol adjacent columns of one pair; thread t -> column t % ncol, line index t / ncol.
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_fwd_cols(const typename cplx_of<T>::type *__restrict__ rowbuf,
           typename cplx_of<T>::type *F, int nb, int lognf, int logc,
           const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, ncol = 1 << logc;
    const int c0 = blockIdx.x << logc, slot = blockIdx.y;
    const int c = threadIdx.x & (ncol - 1), j0 = threadIdx.x >> logc;
    const int tpl = nf >> 4;
    for (int e = j0; e < nf; e += tpl) s[pidx((e << logc) + c)] = mk((T)0, (T)0);
    __syncthreads();
    const C *src = rowbuf + (size_t)slot * nb * nf;
    for (int q = j0; q < nb; q += tpl) {
        const int idx = (q - nb / 2) & (nf - 1);
        s[pidx((idx << logc) + c)] = src[(size_t)q * nf + c0 + c];
    }
    __syncthreads();
    line_fft<C, -1>(s, ncol, c, lognf, j0, tw);
    C *dst = F + (size_t)slot * nf * nf;
    for (int e = j0; e < nf; e += tpl) dst[(size_t)e * nf + c0 + c] = s[pidx((e << logc) + c)];
}

// --------------------------------------------- interpolation / residual / spreading (a3, a4)
// FP32 records: first-tap cell and the fraction f in [0, 1) (the first tap sits at offset
// W/2 - 1 + f from the visibility).
template <int W>
__device__ __forceinline__ void decode(uint2 c, int nf, int &gx, int &gy, float &fx, float &fy) {
    (void)nf;
    gx = (int)(c.x >> FRAC_BITS);
    gy = (int)(c.y >> FRAC_BITS);
    fx = (float)(c.x & (FRAC_ONE - 1)) * (1.0f / (float)FRAC_ONE);
    fy = (float)(c.y & (FRAC_ONE - 1)) * (1.0f / (float)FRAC_ONE);
}
template <int W>
__device__ __forceinline__ void decode(double2 c, int nf, int &gx, int &gy, double &dx, double &dy) {
    const double half = 0.5 * W;
    double g = floor(c.x - half) + 1.0;
    dx = c.x - g;
    gx = (int)g;
    gx = gx < 0 ? gx + nf : gx;
    g = floor(c.y - half) + 1.0;
    dy = c.y - g;
    gy = (int)g;
    gy = gy < 0 ? gy + nf : gy;
}

enum { MODE_COSTGRAD = 0, MODE_PREDICT = 1, MODE_SPREAD = 2 };

// Vector reduction into global memory for one complex cell (sm_90+ has 2-wide float adds).
__device__ __forceinline__ void red_add_c(float2 *p, float2 v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add_c(double2 *p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// One CTA per chunk (a run of visibilities of one tile of one pair). The tile's fine-grid
// patch (tile + W - 1 cells square, wrapped) is staged in shared memory. A group of GS lanes
// (GS = W rounded up to a power of two) handles one visibility at a time: lane r owns kernel
// row r. Each lane evaluates one x and one y kernel value, the x values are exchanged by
// shuffles, the row sums of the interpolation are reduced across the group, and the same 2W
// kernel values serve the spreading. Each group walks a contiguous run of the chunk, whose
// visibilities are sorted by first-tap cell (row-major within each 8 x 8-cell block): a lane
// keeps its row of the spread in registers; while the cell repeats nothing is written, and
// when the next first tap lies d < W cells further right on the same row only the d cells
// that leave the window are added to the shared sub-grid (atomics) before the window slides
// (any other step adds the whole row; adding early is always correct). MODE_PREDICT
// writes V~ to pred[pred_off + orig] instead of spreading; MODE_SPREAD skips the
// interpolation and spreads w times the record's value (the w-stacked entries).
template <typename T, int W, int MODE, int TS = GTILE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 2)
k_grid_pass(const Chunk *__restrict__ chunks, const PairData<T> *__restrict__ pdata,
            const typename cplx_of<T>::type *__restrict__ F, typename cplx_of<T>::type *G,
            int lognf, int ntx, int fhalf, int gfold, T beta, const float *__restrict__ kpoly,
            double *jpart, typename cplx_of<T>::type *pred) {
    typedef typename cplx_of<T>::type C;
    constexpr int GS = W <= 4 ? 4 : (W <= 8 ? 8 : 16);
    constexpr int NG = 256 / GS;  // groups per CTA
    constexpr int tile = TS;
    constexpr int PW = tile + W - 1;
    constexpr bool POLY = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const int nf = 1 << lognf;
    C *Fs = reinterpret_cast<C *>(smem_raw);
    C *Gs = MODE == MODE_SPREAD ? Fs : Fs + PW * PW;  // MODE_SPREAD stages no F tile
    const Chunk ch = chunks[blockIdx.x];
    const PairData<T> pd = pdata[ch.slot];
    const int ty = ch.tile / ntx, tx = ch.tile - ty * ntx;
    const int x0 = tx * tile, y0 = ty * tile;
    const C *Fp = F + (size_t)ch.slot * nf * nf;
    constexpr bool SPREAD = MODE != MODE_PREDICT;
    // with fhalf only the rows 0 .. nf/2 of F are stored: F(gy, gx) = conj F(-gy, -gx)
    for (int i = threadIdx.x; i < PW * PW; i += blockDim.x) {
        const int ly = i / PW, lx = i - ly * PW;
        const int gy = (y0 + ly) & (nf - 1), gx = (x0 + lx) & (nf - 1);
        if (MODE != MODE_SPREAD) {
            if (!fhalf || gy <= nf / 2) {
                Fs[i] = Fp[(size_t)gy * nf + gx];
            } else {
                const C f = Fp[(size_t)(nf - gy) * nf + ((nf - gx) & (nf - 1))];
                Fs[i] = mk(f.x, -f.y);
            }
        }
        if (SPREAD) Gs[i] = mk((T)0, (T)0);
    }
    __syncthreads();
    const T zs = (T)2 / (T)W;
    const int r = threadIdx.x & (GS - 1);  // kernel row of this lane
    const bool active_row = r < W;
    constexpr int KD = es_deg<W>::value;
    float pc[KD + 1];  // this lane's tap polynomial (FP32 path)
#pragma unroll
    for (int i = 0; i <= KD; ++i) pc[i] = (POLY && active_row) ? kpoly[r * (ES_MAXDEG + 1) + i] : 0.f;
    const int len = (ch.end - ch.begin + NG - 1) / NG;  // same for every group of the CTA
    const int vbeg = ch.begin + (threadIdx.x / GS) * len;
    const int vend = min(ch.end, vbeg + len);
    T jacc = (T)0;
    C racc[W];
#pragma unroll
    for (int a = 0; a < W; ++a) racc[a] = mk((T)0, (T)0);
    int clx = -1, cly = 0;  // cell of the run held in racc
    // Every lane of a warp runs exactly len iterations, so the full-warp shuffles below always
    // see all 32 lanes.
    typedef typename coord_of<T>::type CO;
    CO cnext{};  // record of the next visibility, fetched one iteration ahead
    C vnext = mk((T)0, (T)0);
    T wnext = (T)0;
    if (vbeg < vend) {
        cnext = pd.coord[vbeg];
        if (SPREAD) { vnext = pd.vis[vbeg]; wnext = pd.w[vbeg]; }
    }
    for (int i = 0; i < len; ++i) {
        const int v = vbeg + i;
        const bool valid = v < vend;
        const CO ccur = cnext;
        const C vv = vnext;
        const T w = wnext;
        if (v + 1 < vend) {
            cnext = pd.coord[v + 1];
            if (SPREAD) { vnext = pd.vis[v + 1]; wnext = pd.w[v + 1]; }
        }
        int gx = x0, gy = y0;
        T dx = (T)(0.5 * W), dy = (T)(0.5 * W);
        if (valid) decode<W>(ccur, nf, gx, gy, dx, dy);
        const int lx = gx - x0, ly = gy - y0;
        if (SPREAD && valid && (lx != clx || ly != cly)) {
            if (clx >= 0 && active_row) {
                C *gr = Gs + (cly + r) * PW + clx;
                // same kernel-row band, first tap d cells further right (the sort makes d >= 0):
                // only the d leftmost cells of the held row are final. For the common steps of
                // one or two cells those are added and the rest slides along; otherwise the
                // whole row is added (adding early is always correct: the sub-grid sums parts)
                const int d = (ly == cly && lx >= clx) ? lx - clx : W;
                if (d == 1 || d == 2) {
                    atomicAdd(&gr[0].x, racc[0].x);
                    atomicAdd(&gr[0].y, racc[0].y);
                    if (d == 2) {
                        atomicAdd(&gr[1].x, racc[1].x);
                        atomicAdd(&gr[1].y, racc[1].y);
                    }
#pragma unroll
                    for (int a = 0; a < W - 2; ++a) racc[a] = d == 1 ? racc[a + 1] : racc[a + 2];
                    racc[W - 2] = d == 1 ? racc[W - 1] : mk((T)0, (T)0);
                    racc[W - 1] = mk((T)0, (T)0);
                } else {
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        atomicAdd(&gr[a].x, racc[a].x);
                        atomicAdd(&gr[a].y, racc[a].y);
                        racc[a] = mk((T)0, (T)0);
                    }
                }
            }
            clx = lx;
            cly = ly;
        }
        const bool row_on = valid && active_row;
        T kxr, kyr;
        if constexpr (POLY) {
            kxr = row_on ? (T)es_poly<W>(pc, (float)dx) : (T)0;
            kyr = row_on ? (T)es_poly<W>(pc, (float)dy) : (T)0;
        } else {
            kxr = row_on ? es_kernel((dx - (T)r) * zs, beta) : (T)0;
            kyr = row_on ? es_kernel((dy - (T)r) * zs, beta) : (T)0;
        }
        T kx[W];
#pragma unroll
        for (int a = 0; a < W; ++a) kx[a] = __shfl_sync(0xffffffffu, kxr, a, GS);
        C acc = mk((T)0, (T)0);
        if constexpr (MODE != MODE_SPREAD) {
            C row = mk((T)0, (T)0);
            if (row_on) {
                const C *fr = Fs + (ly + r) * PW + lx;
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const C f = fr[a];
                    row.x += kx[a] * f.x;
                    row.y += kx[a] * f.y;
                }
            }
            acc = mk(kyr * row.x, kyr * row.y);
#pragma unroll
            for (int o = GS / 2; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o, GS);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o, GS);
            }
        }
        if (!valid) continue;
        if (MODE == MODE_PREDICT) {
            if (r == 0) pred[pd.pred_off + pd.orig[v]] = acc;
            continue;
        }
        const C res = MODE == MODE_SPREAD ? vv : mk(acc.x - vv.x, acc.y - vv.y);
        // per-visibility term in the working precision; a lane sums at most len (<= 32) terms
        // before the FP64 block and global reductions (FP64 issue is scarce on this part)
        if (MODE == MODE_COSTGRAD && r == 0) jacc += (T)0.5 * w * (res.x * res.x + res.y * res.y);
        if (active_row) {
            const T cyx = kyr * w * res.x, cyy = kyr * w * res.y;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                racc[a].x += cyx * kx[a];
                racc[a].y += cyy * kx[a];
            }
        }
    }
    if (MODE == MODE_PREDICT) return;
    if (clx >= 0 && active_row) {
        C *gr = Gs + (cly + r) * PW + clx;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            atomicAdd(&gr[a].x, racc[a].x);
            atomicAdd(&gr[a].y, racc[a].y);
        }
    }
    if (MODE == MODE_COSTGRAD) {
        double js;
        if constexpr (sizeof(T) == 4) js = block_sum_warpf(jacc, red);  // <= 4 lanes per warp carry terms
        else js = block_sum((double)jacc, red);
        if (threadIdx.x == 0) jpart[blockIdx.x] = js;
    }
    __syncthreads();
    C *Gp = G + (size_t)ch.slot * nf * nf;
    for (int i = threadIdx.x; i < PW * PW; i += blockDim.x) {
        const C g = Gs[i];
        if (g.x == (T)0 && g.y == (T)0) continue;
        const int ly = i / PW, lx = i - ly * PW;
        const int gy = (y0 + ly) & (nf - 1), gx = (x0 + lx) & (nf - 1);
        // gfold: the adjoint uses the Hermitian part of G only, so a row past nf/2 is added,
        // conjugated, to its mirror instead
        if (!gfold || gy <= nf / 2) red_add_c(&Gp[(size_t)gy * nf + gx], g);
        else red_add_c(&Gp[(size_t)(nf - gy) * nf + ((nf - gx) & (nf - 1))], mk(g.x, -g.y));
    }
}

// ---------------------------------------------------------------- adjoint column pass (a5)
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
k_adj_cols(typename cplx_of<T>::type *__restrict__ G,
           typename cplx_of<T>::type *rowbuf, int nb, int lognf, int logc,
           const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, ncol = 1 << logc;
    const int c0 = blockIdx.x << logc, slot = blockIdx.y;
    const int c = threadIdx.x & (ncol - 1), j0 = threadIdx.x >> logc;
    const int tpl = nf >> 4;
    // the adjoint grid is consumed here and left zeroed for the next spreading pass
    C *src = G + (size_t)slot * nf * nf;
    for (int e = j0; e < nf; e += tpl) s[pidx((e << logc) + c)] = src[(size_t)e * nf + c0 + c];
    __syncthreads();
    for (int e = j0; e < nf; e += tpl) src[(size_t)e * nf + c0 + c] = mk((T)0, (T)0);
    line_fft<C, +1>(s, ncol, c, lognf, j0, tw);
    C *dst = rowbuf + (size_t)slot * nb * nf;
    for (int q = j0; q < nb; q += tpl) {
        const int idx = (q - nb / 2) & (nf - 1);
        dst[(size_t)q * nf + c0 + c] = s[pidx((idx << logc) + c)];
    }
}

// ------------------------------------------- adjoint row pass + deapod + Re + beam (a5, a6)
template <typename T>
__global__ void __launch_bounds__(256)
k_adj_rows(const typename cplx_of<T>::type *__restrict__ rowbuf,
           const T *__restrict__ beams, const PairInfo *__restrict__ pinfo,
           const T *__restrict__ dinv, T *contrib, int n, int nb, int lognf,
           const typename cplx_of<T>::type *__restrict__ tw, const T *__restrict__ wx,
           const T *__restrict__ wcorr) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int nf = 1 << lognf, tpl = nf >> 4, lpb = blockDim.x / tpl;
    const int slot = blockIdx.y;
    const PairInfo pi = pinfo[slot];
    const int l = threadIdx.x / tpl, j0 = threadIdx.x - l * tpl;
    const int q = blockIdx.x * lpb + l;
    const int y = pi.cy - nb / 2 + q;
    // rows of an integer window that fall off the sky are never gathered
    const bool on = q < nb && (pi.gridded || (y >= 0 && y < n));
    if (on) {
        const C *src = rowbuf + ((size_t)slot * nb + q) * nf;
        for (int e = j0; e < nf; e += tpl) s[pidx(l * nf + e)] = src[e];
    }
    __syncthreads();
    line_fft<C, +1>(s, 1, l * nf, lognf, j0, tw);
    if (!on) return;
    const T *brow = beams + ((size_t)pi.k * nb + q) * nb;
    const T dq = dinv[q];
    T *out = contrib + ((size_t)slot * nb + q) * nb;
    for (int p = j0; p < nb; p += tpl) {
        const int idx = (p - nb / 2) & (nf - 1);
        const C v = s[pidx(l * nf + idx)];
        T re = v.x;
        if (pi.wplane) {  // Re(corr exp(+2 pi i wk x') v)
            const size_t t = (size_t)q * nb + p;
            T sn, cs;
            sincospi_t((T)(2.0 * pi.wk) * wx[t], &sn, &cs);
            re = (v.x * cs - v.y * sn) * wcorr[t];
        }
        out[p] = re * dinv[p] * dq * brow[p];
    }
}

}  // namespace ivis
