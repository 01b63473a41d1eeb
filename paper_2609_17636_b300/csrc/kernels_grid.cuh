// kernels_grid.cuh -- fused interpolation / residual / J partial / spreading of the FP32 cost
// and gradient evaluation (paper Eqs. 3-6: the type-2 NUFFT for V~, the residual and the
// weighted misfit J_k, and the type-1 NUFFT of w r for the gradient), for kernel widths W <= 8.
//
// One CTA per chunk of the work list: a run of visibilities whose first taps lie in one TS x TS
// tile of one pair's fine grid. The CTA stages the tile's patch of the forward grid F (TS + W - 1
// cells square, wrapped) in shared memory and accumulates the patch of the adjoint grid G there,
// as two planes (real, imaginary), before adding it to global memory with vector reductions.
//
// A group of 8 lanes handles one visibility; lane a owns kernel column a (x tap a):
//   * lane a evaluates the x kernel value of its column and the y kernel value of row a
//     (per-tap polynomials of the ES kernel); the y values are exchanged by shuffles;
//   * interpolation: lane a sums its column, sum_b ky_b F[y + b][x + a], times its x value; the
//     column sums are reduced across the group -> V~;
//   * r = V~ - V, the J term 1/2 w |r|^2 (lane 0), and lane a adds ky_b kx_a w r to the W cells
//     of its column with shared-memory atomics. The W lanes of a group hit W consecutive words
//     of one row of each plane, so a group's atomics never collide with each other.
// Compared with one lane per kernel row, no lane keeps a per-row window of the spread in
// registers, so every lane runs the same straight-line code for every visibility.
#pragma once
#include "common.cuh"
#include "kernels_nufft.cuh"

namespace ivis {

template <int W, int TS>
struct GridCG {
    static constexpr int PW = TS + W - 1;           // patch edge (cells)
    static constexpr int THREADS = TS == 64 ? 512 : 256;
    static constexpr int NG = THREADS / 8;          // visibility groups per CTA
    static constexpr int MINB = TS == 64 ? 2 : 4;   // CTAs per SM the register budget allows
    static constexpr size_t SMEM = (size_t)PW * PW * (sizeof(float2) + 2 * sizeof(float));
};

template <int W, int TS>
__global__ void __launch_bounds__(GridCG<W, TS>::THREADS, GridCG<W, TS>::MINB)
k_grid_cg(const Chunk *__restrict__ chunks, const PairData<float> *__restrict__ pdata,
          const float2 *__restrict__ F, float2 *G, int lognf, const float *__restrict__ kpoly,
          double *jpart) {
    static_assert(W <= 8, "one lane per kernel column in groups of 8");
    typedef GridCG<W, TS> P;
    constexpr int PW = P::PW, NG = P::NG;
    constexpr int KD = es_deg<W>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    float2 *Fs = reinterpret_cast<float2 *>(smem_raw);  // [PW][PW] interleaved
    float *Gr = reinterpret_cast<float *>(Fs + PW * PW); // [PW][PW] real plane
    float *Gi = Gr + PW * PW;                            // [PW][PW] imaginary plane
    const int nf = 1 << lognf, ntx = nf / TS;
    const Chunk ch = chunks[blockIdx.x];
    const PairData<float> pd = pdata[ch.slot];
    const int ty = ch.tile / ntx, tx = ch.tile - ty * ntx;
    const int x0 = tx * TS, y0 = ty * TS;
    const float2 *Fp = F + (size_t)ch.slot * nf * nf;
    // stage F (wrapped) two cells at a time; PW is even for odd W, so pairs never straddle a
    // row, and the wrap point nf - x0 is a multiple of TS
    if constexpr ((PW & 1) == 0) {
        constexpr int PH = PW / 2;
        for (int i = threadIdx.x; i < PW * PH; i += P::THREADS) {
            const int ly = i / PH, lp = i - ly * PH;
            const int gy = (y0 + ly) & (nf - 1), gx = (x0 + 2 * lp) & (nf - 1);
            reinterpret_cast<float4 *>(Fs)[i] = *reinterpret_cast<const float4 *>(Fp + (size_t)gy * nf + gx);
        }
    } else {
        for (int i = threadIdx.x; i < PW * PW; i += P::THREADS) {
            const int ly = i / PW, lx = i - ly * PW;
            Fs[i] = Fp[(size_t)((y0 + ly) & (nf - 1)) * nf + ((x0 + lx) & (nf - 1))];
        }
    }
    for (int i = threadIdx.x; i < PW * PW; i += P::THREADS) {
        Gr[i] = 0.f;
        Gi[i] = 0.f;
    }
    __syncthreads();
    const int a = threadIdx.x & 7;  // kernel column of this lane
    const bool col_on = a < W;
    float pc[KD + 1];
#pragma unroll
    for (int i = 0; i <= KD; ++i) pc[i] = col_on ? kpoly[a * (ES_MAXDEG + 1) + i] : 0.f;
    const int len = (ch.end - ch.begin + NG - 1) / NG;  // the same for every group of the CTA
    const int vbeg = ch.begin + (threadIdx.x >> 3) * len;
    const int vend = min(ch.end, vbeg + len);
    float jacc = 0.f;
    uint2 cnext = make_uint2(0u, 0u);
    float2 vnext = make_float2(0.f, 0.f);
    float wnext = 0.f;
    if (vbeg < vend) {
        cnext = pd.coord[vbeg];
        vnext = pd.vis[vbeg];
        wnext = pd.w[vbeg];
    }
    // every lane of a warp runs exactly len iterations: the width-8 shuffles see all lanes
    for (int i = 0; i < len; ++i) {
        const int v = vbeg + i;
        const bool valid = v < vend;
        const uint2 cc = cnext;
        const float2 vv = vnext;
        const float w = wnext;
        if (v + 1 < vend) {
            cnext = pd.coord[v + 1];
            vnext = pd.vis[v + 1];
            wnext = pd.w[v + 1];
        }
        int gx, gy;
        float fx, fy;
        decode<W>(cc, nf, gx, gy, fx, fy);
        const int lx = gx - x0, ly = gy - y0;  // first tap inside the tile: [0, TS)
        const bool on = valid && col_on;
        const float kxa = on ? es_poly<W>(pc, fx) : 0.f;
        const float kya = on ? es_poly<W>(pc, fy) : 0.f;
        float ky[W];
#pragma unroll
        for (int b = 0; b < W; ++b) ky[b] = __shfl_sync(0xffffffffu, kya, b, 8);
        float2 acc = make_float2(0.f, 0.f);
        const int base = ly * PW + lx + a;
        if (on) {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float2 f = Fs[base + b * PW];
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
        // per-visibility term in FP32; a lane sums at most len terms before the FP64 block and
        // global reductions (FP64 issue is scarce on this part)
        if (valid && a == 0) jacc = fmaf(0.5f * w, rx * rx + ry * ry, jacc);
        if (on) {
            const float s = kxa * w;
            const float cx = s * rx, cy = s * ry;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                atomicAdd(&Gr[base + b * PW], ky[b] * cx);
                atomicAdd(&Gi[base + b * PW], ky[b] * cy);
            }
        }
    }
    const double js = block_sum_warpf(jacc, red);
    if (threadIdx.x == 0) jpart[blockIdx.x] = js;
    __syncthreads();
    float2 *Gp = G + (size_t)ch.slot * nf * nf;
    if constexpr ((PW & 1) == 0) {
        constexpr int PH = PW / 2;
        for (int i = threadIdx.x; i < PW * PH; i += P::THREADS) {
            const float2 re = reinterpret_cast<const float2 *>(Gr)[i];
            const float2 im = reinterpret_cast<const float2 *>(Gi)[i];
            if (re.x == 0.f && re.y == 0.f && im.x == 0.f && im.y == 0.f) continue;
            const int ly = i / PH, lp = i - ly * PH;
            const int gy = (y0 + ly) & (nf - 1), gx = (x0 + 2 * lp) & (nf - 1);
            atomicAdd(reinterpret_cast<float4 *>(Gp + (size_t)gy * nf + gx), make_float4(re.x, im.x, re.y, im.y));
        }
    } else {
        for (int i = threadIdx.x; i < PW * PW; i += P::THREADS) {
            const float re = Gr[i], im = Gi[i];
            if (re == 0.f && im == 0.f) continue;
            const int ly = i / PW, lx = i - ly * PW;
            atomicAdd(Gp + (size_t)((y0 + ly) & (nf - 1)) * nf + ((x0 + lx) & (nf - 1)), make_float2(re, im));
        }
    }
}

}  // namespace ivis
