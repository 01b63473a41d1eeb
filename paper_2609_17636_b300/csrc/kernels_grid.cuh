// kernels_grid.cuh -- fused interpolation / residual / J partial / spreading of the FP32 cost
// and gradient evaluation (paper Eqs. 3-6: the type-2 NUFFT for V~, the residual and the
// weighted misfit J_k, and the type-1 NUFFT of w r for the gradient), for kernel widths W <= 8.
//
// Work list: the visibilities of a pair are sorted by first-tap cell in 8 x 8-cell blocks, and
// an item is a run of at most L visibilities of one block. One CTA takes a chunk: items of one
// TS x TS tile of one pair's fine grid, taken by its NG groups of 8 lanes in rounds (item
// g + k NG in round k; items sorted by length, so the groups of a warp get similar lengths).
//
//   * The CTA stages the tile's patch of the forward grid F (TS + W - 1 cells square,
//     wrapped) in shared memory; with fhalf only rows 0 .. nf/2 of F are stored and a row past
//     nf/2 is read from its mirror, conjugated (F(-k) = conj F(k) for a real window).
//   * Each group owns a private (8 + W - 1)^2 buffer of the adjoint grid for its current
//     item's block (in half lines, see hl_off), so its spreading is a plain
//     read-modify-write: no atomics. Shared-memory
//     float atomics are emulated on this part (a load and a compare-and-swap per value) and
//     cost about four times a plain access, which made them the bound of a spreading pass
//     built on them.
//   * Lane a of a group owns kernel column a: it evaluates the x kernel value of its column
//     and the y value of row a (per-tap polynomials of the ES kernel); the y values are
//     exchanged by shuffles. Interpolation: lane a sums its column of F times the y values,
//     times its x value; the column sums are reduced across the group -> V~. Then r = V~ - V,
//     the J term 1/2 w |r|^2 (lane 0), and lane a adds ky_b kx_a w r to the W cells of its
//     column in the group's buffer.
//   * After each item the group adds its buffer to the global adjoint grid with 16-byte vector
//     reductions (two cells each; neighbouring blocks overlap by W - 1 cells) and clears it.
//     The adjoint passes use only the Hermitian part (G(k) + conj G(-k)) / 2 of each grid, so
//     with gfold a cell in a row past nf/2 is added, conjugated, to its mirror -k instead: the
//     rows past nf/2 stay zero and are neither read nor cleared.
#pragma once
#include "common.cuh"
#include "kernels_nufft.cuh"

namespace ivis {

// One run of visibilities of one 8 x 8-cell block: sorted positions [begin, end) of its pair,
// blk = the block's index within its tile (row-major, TS / 8 blocks per row).
struct Item {
    int begin, end, blk, pad;
};

template <int W, int TS>
struct GridCG {
    static constexpr int PW = TS + W - 1;         // tile patch edge (cells)
    static constexpr int FCELLS = (PW * PW + 1) & ~1;  // F patch cells, even: buffers 16-byte aligned
    static constexpr int BW = 8 + W - 1;          // block buffer edge (cells)
    static constexpr int BWP = BW + (BW & 1);     // buffer row pitch: even, 16-byte cell pairs
    static constexpr int BSEG = (BW * BWP + 7) / 8;  // 8-cell segments of one group buffer
    static constexpr int NBX = TS / 8;            // blocks per tile row
    static constexpr int NG = TS == 64 ? 32 : 16; // groups of 8 lanes
    static constexpr int THREADS = NG * 8;
    static constexpr int MINB = TS == 64 ? 2 : 5;
    static constexpr size_t SMEM = (size_t)FCELLS * sizeof(float2) + (size_t)(NG / 2) * BSEG * 16 * sizeof(float2);
};

// Group buffers in "half lines": buffer cell i (row-major, pitch BWP) of group g sits in half
// g & 1 (64 bytes, 16 banks) of the 128-byte line i / 8 of its group pair, at position i % 8.
// A group's 8 lanes touch 8 consecutive cells, which have distinct positions, so they cover
// exactly their half's banks, and the two groups of a half-warp (served together for 8-byte
// accesses) never meet on a bank: the spreading read-modify-writes are conflict-free.
__device__ __forceinline__ int hl_off(int i) { return i + (i & ~7); }  // float2 offset in the pair's lines

template <int W, int TS>
__global__ void __launch_bounds__(GridCG<W, TS>::THREADS, GridCG<W, TS>::MINB)
k_grid_cg(const Chunk *__restrict__ chunks, const Item *__restrict__ items,
          const PairData<float> *__restrict__ pdata, const float2 *__restrict__ F, float2 *G, int lognf,
          int fhalf, int gfold, const float *__restrict__ kpoly, double *jpart) {
    static_assert(W <= 8, "one lane per kernel column in groups of 8");
    typedef GridCG<W, TS> P;
    constexpr int PW = P::PW, BW = P::BW, BWP = P::BWP, NG = P::NG;
    constexpr int KD = es_deg<W>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    float2 *Fs = reinterpret_cast<float2 *>(smem_raw);   // [PW][PW] tile patch of F
    float2 *buf = Fs + P::FCELLS;                         // [NG/2][BSEG][2][8] group buffers
    const int nf = 1 << lognf, ntx = nf / TS;
    const Chunk ch = chunks[blockIdx.x];  // begin/end: this chunk's items
    const int nitem = ch.end - ch.begin;
    const PairData<float> pd = pdata[ch.slot];
    const int ty = ch.tile / ntx, tx = ch.tile - ty * ntx;
    const int x0 = tx * TS, y0 = ty * TS;
    const float2 *Fp = F + (size_t)ch.slot * nf * nf;
    float2 *Gp = G + (size_t)ch.slot * nf * nf;
    // stage F (wrapped) two cells at a time; PW is even for odd W, so pairs never straddle a
    // row, and the wrap point nf - x0 is a multiple of TS. With fhalf, rows past nf/2 are not
    // stored: F(gy, gx) = conj F(-gy, -gx) (the window is real)
    if constexpr ((PW & 1) == 0) {
        // all of a thread's loads first, then its stores: a mirrored row is read at the mirrored
        // cells and conjugated by a sign, with no branch between the loads
        constexpr int PH = PW / 2;
        constexpr int NIT = (PW * PH + P::THREADS - 1) / P::THREADS;
        float2 f0[NIT], f1[NIT];
        float sg[NIT];
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
            const int i = threadIdx.x + k * P::THREADS;
            f0[k] = f1[k] = make_float2(0.f, 0.f);
            sg[k] = 1.f;
            if (i < PW * PH) {
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
        for (int k = 0; k < NIT; ++k) {
            const int i = threadIdx.x + k * P::THREADS;
            if (i < PW * PH)
                reinterpret_cast<float4 *>(Fs)[i] = make_float4(f0[k].x, sg[k] * f0[k].y, f1[k].x, sg[k] * f1[k].y);
        }
    } else {
        for (int i = threadIdx.x; i < PW * PW; i += P::THREADS) {
            const int ly = i / PW, lx = i - ly * PW;
            const int gy = (y0 + ly) & (nf - 1), gx = (x0 + lx) & (nf - 1);
            if (!fhalf || gy <= nf / 2) {
                Fs[i] = Fp[(size_t)gy * nf + gx];
            } else {
                const float2 f = Fp[(size_t)(nf - gy) * nf + ((nf - gx) & (nf - 1))];
                Fs[i] = make_float2(f.x, -f.y);
            }
        }
    }
    const int g = threadIdx.x >> 3, a = threadIdx.x & 7;
    float2 *B = buf + (size_t)(g >> 1) * P::BSEG * 16 + 8 * (g & 1);  // cell i at B[hl_off(i)]
    for (int l = 0; l < P::BSEG; ++l) B[l * 16 + a] = make_float2(0.f, 0.f);
    __syncthreads();  // F staged, buffers clear
    const bool col_on = a < W;
    float pc[KD + 1];
#pragma unroll
    for (int i = 0; i <= KD; ++i) pc[i] = col_on ? kpoly[a * (ES_MAXDEG + 1) + i] : 0.f;
    float jacc = 0.f;
    const int rounds = (nitem + NG - 1) / NG;  // the same for every group of the CTA
    for (int rd = 0; rd < rounds; ++rd) {
        const int ii = rd * NG + g;
        Item it{0, 0, 0, 0};
        if (ii < nitem) it = items[ch.begin + ii];
        const int n = it.end - it.begin;
        // every lane of a warp runs the same number of iterations: the width-8 shuffles see all
        // lanes
        const int len = __reduce_max_sync(0xffffffffu, n);
        const int ox = (it.blk % P::NBX) * 8, oy = (it.blk / P::NBX) * 8;
        uint2 cnext = make_uint2(0u, 0u);
        float2 vnext = make_float2(0.f, 0.f);
        float wnext = 0.f;
        if (n > 0) {
            cnext = pd.coord[it.begin];
            vnext = pd.vis[it.begin];
            wnext = pd.w[it.begin];
        }
        for (int i = 0; i < len; ++i) {
            const int v = it.begin + i;
            const bool valid = i < n;
            const uint2 cc = cnext;
            const float2 vv = vnext;
            const float w = wnext;
            if (i + 1 < n) {
                cnext = pd.coord[v + 1];
                vnext = pd.vis[v + 1];
                wnext = pd.w[v + 1];
            }
            int gx, gy;
            float fx, fy;
            decode<W>(cc, nf, gx, gy, fx, fy);
            const int lx = gx - x0 - ox, ly = gy - y0 - oy;  // first tap inside the block: [0, 8)
            const bool on = valid && col_on;
            const float kxa = on ? es_poly<W>(pc, fx) : 0.f;
            const float kya = on ? es_poly<W>(pc, fy) : 0.f;
            float ky[W];
#pragma unroll
            for (int b = 0; b < W; ++b) ky[b] = __shfl_sync(0xffffffffu, kya, b, 8);
            float2 acc = make_float2(0.f, 0.f);
            if (on) {
                const float2 *fr = Fs + (oy + ly) * PW + ox + lx + a;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float2 f = fr[b * PW];
                    acc.x = fmaf(ky[b], f.x, acc.x);
                    acc.y = fmaf(ky[b], f.y, acc.y);
                }
            }
            acc.x *= kxa;
            acc.y *= kxa;
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o, 8);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o, 8);
            }
            const float rx = acc.x - vv.x, ry = acc.y - vv.y;
            // per-visibility term in FP32; a lane sums the terms of its group's items before the
            // FP64 block and global reductions (FP64 issue is scarce on this part)
            if (valid && a == 0) jacc = fmaf(0.5f * w, rx * rx + ry * ry, jacc);
            if (on) {
                const float s = kxa * w;
                const float cx = s * rx, cy = s * ry;
                const int i0 = ly * BWP + lx + a;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    float2 *q = B + hl_off(i0 + b * BWP);
                    float2 t = *q;
                    t.x = fmaf(ky[b], cx, t.x);
                    t.y = fmaf(ky[b], cy, t.y);
                    *q = t;
                }
            }
            __syncwarp();  // this visibility's buffer writes before the next one's reads
        }
        // add the block's buffer to the adjoint grid, two cells per vector reduction, and clear
        // it for the next round (pitch BWP is even and x0 + ox is a multiple of 8, so pairs
        // start at even cells: 16-byte aligned in both memories, inside one half line, and
        // never across the grid's wrap). A folded row
        // (gfold, gy past nf/2) goes to row nf - gy conjugated and mirrored: buffer cells
        // (c - 1, c), c even, land on the aligned pair (-(X + c), -(X + c) + 1), X = x0 + ox.
        if (n > 0) {
            constexpr int BH = BWP / 2;                      // pairs of a plain row
            constexpr int BF = (BW - 1 + ((BW - 1) & 1)) / 2 + 1;  // pairs of a folded row
            constexpr int NJ = BH > BF ? BH : BF;
            const int X = x0 + ox;
            for (int i = a; i < BW * NJ; i += 8) {
                const int r = i / NJ, j = i - r * NJ;
                const int gy = (y0 + oy + r) & (nf - 1);
                const int ir = r * BWP;
                if (!gfold || gy <= nf / 2) {
                    if (j >= BH) continue;
                    float4 *q = reinterpret_cast<float4 *>(B + hl_off(ir + 2 * j));
                    const float4 val = *q;
                    *q = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (val.x == 0.f && val.y == 0.f && val.z == 0.f && val.w == 0.f) continue;
                    atomicAdd(reinterpret_cast<float4 *>(Gp + (size_t)gy * nf + ((X + 2 * j) & (nf - 1))), val);
                } else {
                    if (j >= BF) continue;
                    // the adjoint uses only the Hermitian part of G: c at k counts as conj(c) at -k
                    const int c = 2 * j;
                    float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
                    if (c >= 1) {
                        float2 *q0 = B + hl_off(ir + c - 1);
                        v0 = *q0;
                        *q0 = make_float2(0.f, 0.f);
                    }
                    if (c < BW) {
                        float2 *q1 = B + hl_off(ir + c);
                        v1 = *q1;
                        *q1 = make_float2(0.f, 0.f);
                    }
                    if (v0.x == 0.f && v0.y == 0.f && v1.x == 0.f && v1.y == 0.f) continue;
                    atomicAdd(reinterpret_cast<float4 *>(Gp + (size_t)(nf - gy) * nf + ((nf - X - c) & (nf - 1))),
                              make_float4(v1.x, -v1.y, v0.x, -v0.y));
                }
            }
        }
        __syncwarp();  // cleared before the next round's writes
    }
    const double js = block_sum_warpf(jacc, red);
    if (threadIdx.x == 0) jpart[blockIdx.x] = js;
}

}  // namespace ivis
