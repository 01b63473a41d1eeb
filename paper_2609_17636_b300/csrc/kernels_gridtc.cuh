// kernels_gridtc.cuh -- the fused interpolation / residual / J partial / spreading pass of the
// FP32 cost and gradient (paper Eqs. 3-6: the type-2 NUFFT for V~, the residual and the
// weighted misfit J_k, the type-1 NUFFT of w r for the gradient) as small dense contractions on
// the tensor cores, for kernel widths W <= 8.
//
// Same work list as k_grid_cg: the visibilities of a pair are sorted by first-tap cell in 8 x 8
// blocks; an item is a run of at most L visibilities of one block, a CTA takes the items of one
// TS x TS tile. For one block, every visibility's footprint lies in a 16 x 16 patch (first taps
// 0 .. 7, W <= 8 taps), and with ky_j, kx_j the visibility's kernel values written into zero-
// padded 16-vectors (rows, columns of the patch):
//
//   interpolation   V~_j = ky_j^T F kx_j            T = F^T Ky (16 cells x 8 visibilities), then
//                                                   V~_j = kx_j . T_j (reduced across the warp)
//   spreading       G += sum_j (w_j r_j) ky_j kx_j^T  = Ky diag(w r) Kx^T   (16 x 16)
//
// A warp takes one item at a time and its visibilities eight at a time (the n = 8 or k = 8 side
// of mma.m16n8k8): F^T and the block's adjoint patch G stay in registers as mma fragments for the
// whole item, so a visibility costs no shared-memory read-modify-write (the bound of the scalar
// pass, whose 49 taps were each a shared read of F and a read-modify-write of G).
//
// Precision: each product is formed from TF32 parts, a = a_hi + a_lo with a_hi = a rounded to
// TF32 and a_lo = a - a_hi (exact in FP32), as a_hi b_hi + a_hi b_lo + a_lo b_hi (the "3xTF32"
// split of FP32 products), accumulated in FP32. The tensor core reads the top 19 bits of a TF32
// operand, so a_lo enters truncated: with the dropped a_lo b_lo term, the product's relative
// error is below 2^-20, the accuracy of the FP32 scalar pass at the tensor cores' rate.
#pragma once
#include "common.cuh"
#include "kernels_nufft.cuh"
#include "kernels_grid.cuh"

namespace ivis {

template <int W, int TS>
struct GridTC {
    static constexpr int PR = TS + 8;                     // patch rows: every block's 16 rows
    static constexpr int FP = (TS + 8) + ((12 - (TS + 8) % 16 + 16) % 16);  // row pitch (cells), = 12 mod 16
    static constexpr int NW = 4;                          // warps per CTA
    static constexpr int THREADS = NW * 32;
    static constexpr int MINB = 4;                        // CTAs per SM: at most 128 registers
    static constexpr int KS = 20;                         // row stride of the tap matrices (elements)
    // per warp: Ky as TF32 (hi, lo) pairs [8][KS] (uint2), Kx [8][KS] (float), w r [8] (float2)
    static constexpr int WSCR = 2 * 8 * KS + 8 * KS + 16;  // 32-bit words
    static constexpr size_t SMEM = (size_t)PR * FP * sizeof(float2) + (size_t)NW * WSCR * sizeof(float);
};

// a = hi + lo: hi = a rounded to TF32 (to nearest, ties away from zero: half an ulp of the
// 10-bit mantissa added to the magnitude's bits, the low 13 bits cleared), lo = a - hi, exact
__device__ __forceinline__ void tf32_split(float a, uint32_t &hi, uint32_t &lo) {
    const uint32_t h = (__float_as_uint(a) + 0x1000u) & 0xffffe000u;
    hi = h;
    lo = __float_as_uint(a - __uint_as_float(h));
}

// d += a b, one m16n8k8 TF32 product with FP32 accumulation
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// d = a b, one m16n8k8 TF32 product (zero accumulator)
__device__ __forceinline__ void mma_tf32_0(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                           uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.f));
}

// d = a b in split TF32 (as mma_3xtf32, from a zero accumulator)
__device__ __forceinline__ void mma_3xtf32_0(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                             uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32_0(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

// d += a b in split TF32: the two small cross terms first, then the large one
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

// Fragment coordinates (PTX mma.m16n8k8, .tf32): lane = 4 g + t; A (16 x 8, row): a0 (g, t),
// a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4); B (8 x 8, col): b0 (t, g), b1 (t + 4, g);
// C (16 x 8): c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
template <int W, int TS>
__global__ void __launch_bounds__(GridTC<W, TS>::THREADS, GridTC<W, TS>::MINB)
k_grid_tc(const Chunk *__restrict__ chunks, const Item *__restrict__ items,
          const PairData<float> *__restrict__ pdata, const float2 *__restrict__ F, float2 *G, int lognf,
          int fhalf, int gfold, const float *__restrict__ kpoly, double *jpart) {
    static_assert(W <= 8, "footprints of an 8 x 8 block within 16 x 16 cells");
    typedef GridTC<W, TS> P;
    constexpr int FP = P::FP, KS = P::KS;
    constexpr int KD = es_deg<W>::value;
    constexpr int BW = 8 + W - 1;  // rows / columns of a block's footprint
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    float2 *Fs = reinterpret_cast<float2 *>(smem_raw);  // [PR][FP] tile patch of F
    const int nf = 1 << lognf, ntx = nf / TS;
    const Chunk ch = chunks[blockIdx.x];
    const int nitem = ch.end - ch.begin;
    const PairData<float> pd = pdata[ch.slot];
    const int ty = ch.tile / ntx, tx = ch.tile - ty * ntx;
    const int x0 = tx * TS, y0 = ty * TS;
    const float2 *Fp = F + (size_t)ch.slot * nf * nf;
    float2 *Gp = G + (size_t)ch.slot * nf * nf;
    // stage F (wrapped) two cells at a time: TS + 8 is even and the wrap point nf - x0 is a
    // multiple of TS, so pairs never straddle a row end or the wrap. With fhalf, rows past nf/2
    // are not stored: F(gy, gx) = conj F(-gy, -gx) (the window is real)
    {   // all of a thread's loads first, then its stores (a mirrored row: mirrored cells, sign)
        constexpr int PH = (TS + 8) / 2;
        constexpr int NIT = (P::PR * PH + P::THREADS - 1) / P::THREADS;
#pragma unroll
        for (int k0 = 0; k0 < NIT; k0 += 8) {
            float2 f0[8], f1[8];
            float sg[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = threadIdx.x + (k0 + k) * P::THREADS;
                f0[k] = f1[k] = make_float2(0.f, 0.f);
                sg[k] = 1.f;
                if (k0 + k < NIT && i < P::PR * PH) {
                    const int ly = i / PH, lp = i - ly * PH;
                    const int gy = (y0 + ly) & (nf - 1), gx = (x0 + 2 * lp) & (nf - 1);
                    const bool mir = fhalf && gy > nf / 2;
                    const float2 *row = Fp + (size_t)(mir ? nf - gy : gy) * nf;
                    f0[k] = row[mir ? (nf - gx) & (nf - 1) : gx];
                    f1[k] = row[mir ? (nf - gx - 1) & (nf - 1) : gx + 1];
                    sg[k] = mir ? -1.f : 1.f;
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = threadIdx.x + (k0 + k) * P::THREADS;
                if (k0 + k < NIT && i < P::PR * PH) {
                    const int ly = i / PH, lp = i - ly * PH;
                    *reinterpret_cast<float4 *>(Fs + ly * FP + 2 * lp) =
                        make_float4(f0[k].x, sg[k] * f0[k].y, f1[k].x, sg[k] * f1[k].y);
                }
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    uint32_t *scr = reinterpret_cast<uint32_t *>(smem_raw + (size_t)P::PR * FP * sizeof(float2)) + warp * P::WSCR;
    uint2 *Ky = reinterpret_cast<uint2 *>(scr);               // [8][KS] TF32 (hi, lo)
    float *Kx = reinterpret_cast<float *>(scr + 2 * 8 * KS);  // [8][KS]
    float2 *cws = reinterpret_cast<float2 *>(scr + 3 * 8 * KS);
    // lane t evaluates taps t and t + 4 of its quad's visibility
    const bool ta = t < W, tb = t + 4 < W;
    float pa[KD + 1], pb[KD + 1];
#pragma unroll
    for (int i = 0; i <= KD; ++i) {
        pa[i] = ta ? kpoly[t * (ES_MAXDEG + 1) + i] : 0.f;
        pb[i] = tb ? kpoly[(t + 4) * (ES_MAXDEG + 1) + i] : 0.f;
    }
    const bool rlane = t == (g >> 1);  // this lane forms visibility g's residual
    __syncthreads();  // F staged
    float jacc = 0.f;
    // software pipeline over the warp's items: the next item's descriptor is fetched when an
    // item starts, and the record of visibility g of the next batch (of this item, or the next
    // item's first) one batch ahead, so no global load latency sits at a batch's start
    Item itn{0, 0, 0, 0};
    if (warp < nitem) itn = items[ch.begin + warp];
    uint2 cn = make_uint2(0u, 0u);
    float2 vn = make_float2(0.f, 0.f);
    float wn = 0.f;
    if (itn.begin + g < itn.end) {
        cn = pd.coord[itn.begin + g];
        if (rlane) {
            vn = pd.vis[itn.begin + g];
            wn = pd.w[itn.begin + g];
        }
    }
    for (int ii = warp; ii < nitem; ii += P::NW) {
        const Item it = itn;
        if (ii + P::NW < nitem) itn = items[ch.begin + ii + P::NW];
        else itn = Item{0, 0, 0, 0};
        const int ox = (it.blk % (TS / 8)) * 8, oy = (it.blk / (TS / 8)) * 8;
        // F^T of the block's 16 x 16 patch as A fragments (cells x rows), split into TF32 parts
        uint32_t frh[2][4], frl[2][4], fih[2][4], fil[2][4];
        {
            const float2 *fb = Fs + oy * FP + ox;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float2 f0 = fb[(t + 8 * s) * FP + g], f1 = fb[(t + 8 * s) * FP + g + 8];
                const float2 f2 = fb[(t + 4 + 8 * s) * FP + g], f3 = fb[(t + 4 + 8 * s) * FP + g + 8];
                tf32_split(f0.x, frh[s][0], frl[s][0]);
                tf32_split(f1.x, frh[s][1], frl[s][1]);
                tf32_split(f2.x, frh[s][2], frl[s][2]);
                tf32_split(f3.x, frh[s][3], frl[s][3]);
                tf32_split(f0.y, fih[s][0], fil[s][0]);
                tf32_split(f1.y, fih[s][1], fil[s][1]);
                tf32_split(f2.y, fih[s][2], fil[s][2]);
                tf32_split(f3.y, fih[s][3], fil[s][3]);
            }
        }
        // the block's adjoint patch: rows g, g + 8 x cells 8 nt + 2t, + 1 (C fragments)
        float gre[2][4], gim[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) gre[nt][i] = gim[nt][i] = 0.f;
        for (int base = it.begin; base < it.end; base += 8) {
            // ---- quad g: visibility base + g; its kernel values into row g of Ky, Kx
            const bool valid = base + g < it.end;
            const uint2 cc = cn;
            const float2 vv = vn;
            const float w = wn;
            {
                const bool more = base + 8 < it.end;  // warp-uniform
                const int vnx = more ? base + 8 + g : itn.begin + g;
                if (vnx < (more ? it.end : itn.end)) {
                    cn = pd.coord[vnx];
                    if (rlane) {
                        vn = pd.vis[vnx];
                        wn = pd.w[vnx];
                    }
                }
            }
            int gx, gy;
            float fx, fy;
            decode<W>(cc, nf, gx, gy, fx, fy);
            const int lx = valid ? gx - x0 - ox : 0, ly = valid ? gy - y0 - oy : 0;  // [0, 8)
            const float kya = (valid && ta) ? es_poly<W>(pa, fy) : 0.f;
            const float kyb = (valid && tb) ? es_poly<W>(pb, fy) : 0.f;
            const float kxa = (valid && ta) ? es_poly<W>(pa, fx) : 0.f;
            const float kxb = (valid && tb) ? es_poly<W>(pb, fx) : 0.f;
            // position p = t + 4i of the padded vector holds tap p - l, which lane (p - l) & 3 of
            // the quad evaluated (its first tap if p - l < 4, else its second): with
            // q = (t - l + 8) / 4, the first taps land at i = 2 - q, the second at i = 3 - q
            const float ya = __shfl_sync(0xffffffffu, kya, (lane & ~3) | ((t - ly) & 3));
            const float yb = __shfl_sync(0xffffffffu, kyb, (lane & ~3) | ((t - ly) & 3));
            const float xa = __shfl_sync(0xffffffffu, kxa, (lane & ~3) | ((t - lx) & 3));
            const float xb = __shfl_sync(0xffffffffu, kxb, (lane & ~3) | ((t - lx) & 3));
            const int qy = (t - ly + 8) >> 2, qx = (t - lx + 8) >> 2;
            float ky[4], kx[4];
            ky[0] = qy == 2 ? ya : 0.f;
            ky[1] = qy == 2 ? yb : (qy == 1 ? ya : 0.f);
            ky[2] = qy == 1 ? yb : (qy == 0 ? ya : 0.f);
            ky[3] = qy == 0 ? yb : 0.f;
            kx[0] = qx == 2 ? xa : 0.f;
            kx[1] = qx == 2 ? xb : (qx == 1 ? xa : 0.f);
            kx[2] = qx == 1 ? xb : (qx == 0 ? xa : 0.f);
            kx[3] = qx == 0 ? xb : 0.f;
            // ky[i] is row t + 4i of visibility g: this lane's B fragment of the interpolation
            uint32_t yh[4], yl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                tf32_split(ky[i], yh[i], yl[i]);
                Ky[g * KS + t + 4 * i] = make_uint2(yh[i], yl[i]);
                Kx[g * KS + t + 4 * i] = kx[i];
            }
            // ---- interpolation: T = F^T Ky (cells x visibilities); one accumulator per k step
            float tre[2][4], tim[2][4];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                mma_3xtf32_0(tre[s], frh[s], frl[s], yh[2 * s], yh[2 * s + 1], yl[2 * s], yl[2 * s + 1]);
                mma_3xtf32_0(tim[s], fih[s], fil[s], yh[2 * s], yh[2 * s + 1], yl[2 * s], yl[2 * s + 1]);
            }
            __syncwarp();  // Ky, Kx of all eight visibilities stored
            // V~_j = sum over cells of kx_j T_j: this lane holds cells g, g + 8 of visibilities
            // 2t, 2t + 1; the sum over g runs across the lanes t + 4 g'
            float v0x, v0y, v1x, v1y;
            {
                const float k00 = Kx[(2 * t) * KS + g], k01 = Kx[(2 * t) * KS + g + 8];
                const float k10 = Kx[(2 * t + 1) * KS + g], k11 = Kx[(2 * t + 1) * KS + g + 8];
                v0x = fmaf(k00, tre[0][0] + tre[1][0], k01 * (tre[0][2] + tre[1][2]));
                v0y = fmaf(k00, tim[0][0] + tim[1][0], k01 * (tim[0][2] + tim[1][2]));
                v1x = fmaf(k10, tre[0][1] + tre[1][1], k11 * (tre[0][3] + tre[1][3]));
                v1y = fmaf(k10, tim[0][1] + tim[1][1], k11 * (tim[0][3] + tim[1][3]));
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                v0x += __shfl_xor_sync(0xffffffffu, v0x, o);
                v0y += __shfl_xor_sync(0xffffffffu, v0y, o);
                v1x += __shfl_xor_sync(0xffffffffu, v1x, o);
                v1y += __shfl_xor_sync(0xffffffffu, v1y, o);
            }
            // ---- residual of visibility g (its quad's lane t = g / 2 holds V~_g): r = V~ - V,
            // the J term 1/2 w |r|^2, and w r for the spreading
            if (rlane) {
                float2 cw = make_float2(0.f, 0.f);
                if (valid) {
                    const float rx = ((g & 1) ? v1x : v0x) - vv.x, ry = ((g & 1) ? v1y : v0y) - vv.y;
                    jacc = fmaf(0.5f * w, rx * rx + ry * ry, jacc);
                    cw = make_float2(w * rx, w * ry);
                }
                cws[g] = cw;
            }
            __syncwarp();
            // ---- spreading: G += Ky diag(w r) Kx^T (rows x cells; k = the 8 visibilities)
            {
                const uint2 y0 = Ky[t * KS + g], y1 = Ky[t * KS + g + 8];
                const uint2 y2 = Ky[(t + 4) * KS + g], y3 = Ky[(t + 4) * KS + g + 8];
                const uint32_t ah[4] = {y0.x, y1.x, y2.x, y3.x}, al[4] = {y0.y, y1.y, y2.y, y3.y};
                const float2 c0 = cws[t], c1 = cws[t + 4];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const float k0 = Kx[t * KS + g + 8 * nt], k1 = Kx[(t + 4) * KS + g + 8 * nt];
                    uint32_t h0, l0, h1, l1;
                    tf32_split(c0.x * k0, h0, l0);
                    tf32_split(c1.x * k1, h1, l1);
                    mma_3xtf32(gre[nt], ah, al, h0, h1, l0, l1);
                    tf32_split(c0.y * k0, h0, l0);
                    tf32_split(c1.y * k1, h1, l1);
                    mma_3xtf32(gim[nt], ah, al, h0, h1, l0, l1);
                }
            }
            __syncwarp();  // this batch's reads of Ky, Kx, w r before the next batch's writes
        }
        // ---- add the block's patch to the adjoint grid: this lane holds rows g, g + 8 x cells
        // (c, c + 1), c = 8 nt + 2t, a 16-byte pair in both memories (x0 + ox is a multiple of 8;
        // pairs never cross the grid's wrap). With gfold a row past nf/2 goes, conjugated, to
        // row nf - gy and mirrored columns: the aligned mirrored pair is cells (c - 1, c), whose
        // first cell the lane t - 1 (t = 0: lane 3, previous nt) holds as its second
        float pre[2][2], pim[2][2];  // cell c - 1 for [nt][row half]
        if (gfold) {
            const int src = (lane & ~3) | ((t + 3) & 3);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const float r0 = __shfl_sync(0xffffffffu, gre[nt][1], src), i0 = __shfl_sync(0xffffffffu, gim[nt][1], src);
                const float r1 = __shfl_sync(0xffffffffu, gre[nt][3], src), i1 = __shfl_sync(0xffffffffu, gim[nt][3], src);
                pre[nt][0] = r0; pim[nt][0] = i0; pre[nt][1] = r1; pim[nt][1] = i1;
            }
            if (t == 0) {  // cell 8 nt - 1: the previous nt's last cell; none before cell 0
                pre[1][0] = pre[0][0]; pim[1][0] = pim[0][0]; pre[1][1] = pre[0][1]; pim[1][1] = pim[0][1];
                pre[0][0] = pim[0][0] = pre[0][1] = pim[0][1] = 0.f;
            }
        }
        const int X = x0 + ox;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = g + 8 * h;
            if (r >= BW) continue;
            const int gyr = (y0 + oy + r) & (nf - 1);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int c = 8 * nt + 2 * t;
                if (!gfold || gyr <= nf / 2) {
                    if (c >= BW) continue;  // cells c, c + 1 past the footprint: zero
                    const float4 val = make_float4(gre[nt][2 * h], gim[nt][2 * h], gre[nt][2 * h + 1], gim[nt][2 * h + 1]);
                    atomicAdd(reinterpret_cast<float4 *>(Gp + (size_t)gyr * nf + ((X + c) & (nf - 1))), val);
                } else {
                    // cells (c - 1, c) -> (-(X + c) + 1, -(X + c)) conjugated: stored as the pair
                    // starting at -(X + c)
                    const float4 val = make_float4(gre[nt][2 * h], -gim[nt][2 * h], pre[nt][h], -pim[nt][h]);
                    atomicAdd(reinterpret_cast<float4 *>(Gp + (size_t)(nf - gyr) * nf + ((nf - X - c) & (nf - 1))), val);
                }
            }
        }
    }
    const double js = block_sum_warpf(jacc, red);
    if (threadIdx.x == 0) jpart[blockIdx.x] = js;
}

}  // namespace ivis
