// kernels_unet.cuh -- kernels of the learned warm start (a U-Net mapping [dirty image,
// beam-weight map] to an initial sky).
//
// Convolutions are lowered to GEMMs: an im2col gather (which also folds in the nearest-
// neighbour 2x upsampling and the channel concatenation of the decoder inputs) followed by a
// BF16 tensor-core GEMM with FP32 accumulation: tcgen05 (TMEM accumulators) for the forward
// convolutions and the parameter gradients, mma.sync m16n8k16 for the activation gradients
// (and for everything when tcgen05 is switched off). Activations are NHWC BF16; activation
// gradients are FP32 and are rounded to BF16 only as GEMM operands; weights are FP32 masters
// with BF16 copies; Adam runs in FP32.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace ivis {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------------------- GEMM
// C[M x N] = op(A) op(B) with A given either as [M][K] (TA = 0) or as [K][M] (TA = 1),
// B either as [K][N] (TB = 0) or [N][K] (TB = 1), all row-major BF16. Split-K over gridDim.z.
// EPI 0: C bf16 = relu?(acc + bias[n]) ; EPI 1: C fp32 = acc ; EPI 2: C fp32 += acc (atomic).
constexpr int GB_M = 128, GB_N = 64, GB_K = 32, GB_PAD = 8;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int TA, int TB, int EPI>
__global__ void __launch_bounds__(256)
k_gemm_bf16(int M, int N, int K, int kchunk, const bf16 *__restrict__ A, const bf16 *__restrict__ B,
            void *Cout, const float *__restrict__ bias, int relu) {
    __shared__ __align__(16) bf16 As[GB_M][GB_K + GB_PAD];
    __shared__ __align__(16) bf16 Bs[GB_N][GB_K + GB_PAD];
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // 4 x 2 warps, 32 x 32 each
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    // 16-byte staging when the contiguous dimension of each operand is a multiple of 8
    // (split-K chunk ends are multiples of GB_K, so a vector never straddles kend)
    const bool vecA = TA == 0 ? (K % 8 == 0) : (M % 8 == 0);
    const bool vecB = TB == 1 ? (K % 8 == 0) : (N % 8 == 0);
    for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
        // stage A tile [GB_M][GB_K] (m-major) and B tile [GB_N][GB_K] (n-major)
        if (vecA) {
            for (int v = tid; v < GB_M * GB_K / 8; v += 256) {
                uint4 q = make_uint4(0u, 0u, 0u, 0u);
                if (TA == 0) {
                    const int mm = v / (GB_K / 8), kk = (v % (GB_K / 8)) * 8;
                    const int gm = m0 + mm, gk = k0 + kk;
                    if (gm < M && gk < kend) q = *reinterpret_cast<const uint4 *>(A + (size_t)gm * K + gk);
                    *reinterpret_cast<uint4 *>(&As[mm][kk]) = q;
                } else {
                    const int kk = v / (GB_M / 8), mm = (v % (GB_M / 8)) * 8;
                    const int gm = m0 + mm, gk = k0 + kk;
                    if (gm < M && gk < kend) q = *reinterpret_cast<const uint4 *>(A + (size_t)gk * M + gm);
                    const bf16 *e = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
                    for (int t = 0; t < 8; ++t) As[mm + t][kk] = e[t];
                }
            }
        } else {
            for (int i = tid; i < GB_M * GB_K; i += 256) {
                int mm, kk;
                if (TA == 0) { mm = i / GB_K; kk = i - mm * GB_K; } else { kk = i / GB_M; mm = i - kk * GB_M; }
                const int gm = m0 + mm, gk = k0 + kk;
                bf16 v = zero;
                if (gm < M && gk < kend) v = TA == 0 ? A[(size_t)gm * K + gk] : A[(size_t)gk * M + gm];
                As[mm][kk] = v;
            }
        }
        if (vecB) {
            for (int v = tid; v < GB_N * GB_K / 8; v += 256) {
                uint4 q = make_uint4(0u, 0u, 0u, 0u);
                if (TB == 1) {
                    const int nn = v / (GB_K / 8), kk = (v % (GB_K / 8)) * 8;
                    const int gn = n0 + nn, gk = k0 + kk;
                    if (gn < N && gk < kend) q = *reinterpret_cast<const uint4 *>(B + (size_t)gn * K + gk);
                    *reinterpret_cast<uint4 *>(&Bs[nn][kk]) = q;
                } else {
                    const int kk = v / (GB_N / 8), nn = (v % (GB_N / 8)) * 8;
                    const int gn = n0 + nn, gk = k0 + kk;
                    if (gn < N && gk < kend) q = *reinterpret_cast<const uint4 *>(B + (size_t)gk * N + gn);
                    const bf16 *e = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
                    for (int t = 0; t < 8; ++t) Bs[nn + t][kk] = e[t];
                }
            }
        } else {
            for (int i = tid; i < GB_N * GB_K; i += 256) {
                int nn, kk;
                if (TB == 1) { nn = i / GB_K; kk = i - nn * GB_K; } else { kk = i / GB_N; nn = i - kk * GB_N; }
                const int gn = n0 + nn, gk = k0 + kk;
                bf16 v = zero;
                if (gn < N && gk < kend) v = TB == 1 ? B[(size_t)gn * K + gk] : B[(size_t)gk * N + gn];
                Bs[nn][kk] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GB_K; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
            const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm + i * 16 + r;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[row][ks + c]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[row + 8][ks + c]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[row][ks + c + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[row + 8][ks + c + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = wn + j * 8 + r;
                bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[col][ks + c]);
                bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[col][ks + c + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gm = m0 + wm + i * 16 + r + h * 8;
                if (gm >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int gn = n0 + wn + j * 8 + c + e;
                    if (gn >= N) continue;
                    float v = acc[i][j][h * 2 + e];
                    if (EPI == 0) {
                        v += bias ? bias[gn] : 0.f;
                        if (relu) v = fmaxf(v, 0.f);
                        reinterpret_cast<bf16 *>(Cout)[(size_t)gm * N + gn] = __float2bfloat16(v);
                    } else if (EPI == 1) {
                        reinterpret_cast<float *>(Cout)[(size_t)gm * N + gn] = v;
                    } else {
                        atomicAdd(&reinterpret_cast<float *>(Cout)[(size_t)gm * N + gn], v);
                    }
                }
            }
}

// ------------------------------------------------------------------------- tcgen05 GEMM
// acc[M x N] = A[M x K] B[N x K]^T, both operands K-major bf16 (row stride K), FP32
// accumulation in tensor memory; EPI 0: C bf16 [M][N] = relu?(acc + bias) (forward
// convolutions, stored through shared memory so that a store covers two rows of 16 columns);
// EPI 2: C fp32 [N][M] += acc (parameter gradients, atomic and coalesced along M: the K range
// is split over gridDim.z in chunks of kchunk). One CTA of 4 warps per 128 x BN output tile. The K loop moves
// 128 x 64 slices of A and BN x 64 slices of B into shared memory with 16-byte cp.async copies
// (zero-filled past the edges) in the canonical no-swizzle layout (8-row x 16-byte core
// matrices; core matrices adjacent in K are LBO bytes apart, adjacent in M/N 128 bytes apart),
// TC_STAGES(BN) slices in flight: while the tensor cores work on slice k, the copies of the
// next slices are outstanding. One thread issues four tcgen05.mma (K = 16 each) per slice and
// tcgen05.commit signals that stage's mbarrier; a stage is refilled only after its barrier
// (bounded wait). Operands whose K is not a multiple of 8 (the first layer) are staged through
// registers. The epilogue reads the accumulator rows with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = tile rows) and, per EPI (below), adds the bias, applies the ReLU and stores
// bf16, or reduces into the fp32 parameter gradient.
constexpr int TC_BM = 128, TC_BK = 64;
template <int BN> struct tc_stages { static constexpr int value = BN <= 64 ? 4 : 3; };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    // start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29), stride byte offset
    // >> 4 (32-45), descriptor version 1 (bit 46), no swizzle (bits 61-63 = 0)
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Geometry of an implicit-GEMM 3x3 'same' convolution (the A operand gathered on the fly in
// the im2col order of k_im2col, nothing materialised): output H x W per image, sources a
// (ca channels at H/ua x W/ua, nearest upsampling) and b (cb channels at H x W), NHWC bf16,
// channel counts multiples of 8.
struct ConvGeom {
    const bf16 *a;
    const bf16 *b;
    int ca, ua, cb, H, W;
};

template <int BN, bool IMPLICIT, int EPI>
__global__ void __launch_bounds__(128)
k_gemm_tc(int M, int N, int K, int kchunk, const bf16 *__restrict__ A, const bf16 *__restrict__ B,
          void *C, const float *__restrict__ bias, int relu, int *err, ConvGeom cg) {
    static_assert(EPI == 0 || EPI == 2, "bf16 forward output or fp32 parameter-gradient reduction");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int S = tc_stages<BN>::value;
    constexpr int STAGE = (TC_BM + BN) * TC_BK;  // bf16 elements per stage (A then B)
    bf16 *stage0 = reinterpret_cast<bf16 *>(smem_raw);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stage0 + S * STAGE);  // one per stage
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(mbar + S);
    constexpr int NCOL = BN < 32 ? 32 : BN;  // TMEM columns (power of 2)
    constexpr uint32_t LBO_A = (TC_BM / 8) * 128, LBO_B = (BN / 8) * 128;
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(TC_BM >> 4) << 24);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_holder)), "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < S; ++st) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar + st)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_holder;
    const bool vec = (K % 8) == 0;
    // this CTA's K range (kchunk is a multiple of TC_BK; the whole of K without a split)
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int nk = (kend - kbeg + TC_BK - 1) / TC_BK;
    uint32_t phase[S];
    bool pending[S];
#pragma unroll
    for (int st = 0; st < S; ++st) {
        phase[st] = 0u;
        pending[st] = false;
    }
    // this thread's bounded waits ran out (combined across the CTA at every barrier, so all
    // threads take the same branches and reach the same barriers)
    int fail = 0;
    // bounded wait on stage st's barrier (about two seconds at most); a stage whose wait ran
    // out stays pending, so the drain below waits for it again before tensor memory is freed
    auto wait_stage = [&](int st) -> bool {
        uint32_t done = 0;
        const long long t_start = clock64();
        while (!done) {
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(mbar + st)), "r"(phase[st]));
            if (!done && clock64() - t_start > 4000000000LL) break;
        }
        if (!done) {
            fail = 1;
            if (err) atomicExch(err, 1);
            return false;
        }
        phase[st] ^= 1u;
        pending[st] = false;
        return true;
    };
    // implicit GEMM: this thread always copies chunk kg = tid % 8 of the tile rows
    // tid / 8 + 16 i; their pixel coordinates are fixed for the whole K loop
    int pn[8], pyx[8];
    if constexpr (IMPLICIT) {
        const int HW = cg.H * cg.W;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int pidx_ = m0 + (tid >> 3) + 16 * i;
            const int nimg = pidx_ / HW, rem = pidx_ - nimg * HW, yy = rem / cg.W;
            pn[i] = pidx_ < M ? nimg : -1;
            pyx[i] = (yy << 16) | (rem - yy * cg.W);
        }
    }
    // copies of slice kb into stage st (asynchronous when K is a multiple of 8)
    auto load_slice = [&](int kb, int st) {
        bf16 *As = stage0 + st * STAGE, *Bs = As + TC_BM * TC_BK;
        const int k0 = kbeg + kb * TC_BK;
        if constexpr (IMPLICIT) {
            const int kg = tid & 7, kglob = k0 + kg * 8, cin = cg.ca + cg.cb;
            const bool kin = kglob < kend;
            const int tap = kin ? kglob / cin : 0, ci = kglob - tap * cin;
            const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
            const int Ha = cg.H / cg.ua, Wa = cg.W / cg.ua;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = (tid >> 3) + 16 * i;
                const int yy = (pyx[i] >> 16) + dy, xx = (pyx[i] & 0xFFFF) + dx;
                const bool in = kin && pn[i] >= 0 && yy >= 0 && yy < cg.H && xx >= 0 && xx < cg.W;
                const bf16 *g = cg.b ? cg.b : cg.a;
                if (in) {
                    g = ci < cg.ca
                            ? cg.a + (((size_t)pn[i] * Ha + yy / cg.ua) * Wa + xx / cg.ua) * cg.ca + ci
                            : cg.b + (((size_t)pn[i] * cg.H + yy) * cg.W + xx) * cg.cb + (ci - cg.ca);
                }
                unsigned char *dst = reinterpret_cast<unsigned char *>(As) + kg * LBO_A + (row >> 3) * 128 +
                                     (row & 7) * 16;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             :: "r"(smem_u32(dst)), "l"(g), "r"(in ? 16 : 0));
            }
        }
        for (int v = (IMPLICIT ? TC_BM * (TC_BK / 8) : 0) + tid; v < (TC_BM + BN) * (TC_BK / 8); v += 128) {
            const bool isA = v < TC_BM * (TC_BK / 8);
            const int vv = isA ? v : v - TC_BM * (TC_BK / 8);
            const int row = vv / (TC_BK / 8), kg = vv % (TC_BK / 8);
            const int grow = (isA ? m0 : n0) + row, gk = k0 + kg * 8;
            const int rows = isA ? M : N;
            const bf16 *src = isA ? A : B;
            const uint32_t lbo = isA ? LBO_A : LBO_B;
            unsigned char *dst = reinterpret_cast<unsigned char *>(isA ? As : Bs) + kg * lbo +
                                 (row >> 3) * 128 + (row & 7) * 16;
            if (vec) {
                const bool in = grow < rows && gk < kend;
                const bf16 *g = in ? src + (size_t)grow * K + gk : src;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             :: "r"(smem_u32(dst)), "l"(g), "r"(in ? 16 : 0));
            } else {
                uint4 q = make_uint4(0u, 0u, 0u, 0u);
                if (grow < rows) {
                    bf16 *e = reinterpret_cast<bf16 *>(&q);
                    for (int t = 0; t < 8; ++t)
                        if (gk + t < kend) e[t] = src[(size_t)grow * K + gk + t];
                }
                *reinterpret_cast<uint4 *>(dst) = q;
            }
        }
    };
    // prologue: slices 0 .. S - 2 in flight (one commit group per slice, empty ones included)
#pragma unroll
    for (int s0 = 0; s0 < S - 1; ++s0) {
        if (s0 < nk) load_slice(s0, s0);
        asm volatile("cp.async.commit_group;");
    }
    for (int kb = 0; kb < nk; ++kb) {
        const int st = kb % S;
        asm volatile("cp.async.wait_group %0;" :: "n"(S - 2));  // slice kb has landed
        asm volatile("fence.proxy.async.shared::cta;");
        // one barrier per slice; a wait that ran out in any thread stops all of them here
        if (__syncthreads_or(fail)) break;
        if (tid == 0) {
            bf16 *As = stage0 + st * STAGE, *Bs = As + TC_BM * TC_BK;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = umma_desc(smem_u32(As) + kk * 2 * LBO_A, LBO_A, 128);
                const uint64_t bd = umma_desc(smem_u32(Bs) + kk * 2 * LBO_B, LBO_B, 128);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    :: "r"(tmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mbar + st)));
        }
        pending[st] = true;
        // refill the stage of slice kb - 1 with slice kb + S - 1 once its MMAs are done (not
        // after a wait that ran out: its MMAs may still read it)
        const int nxt = kb + S - 1;
        if (nxt < nk) {
            const int sn = nxt % S;
            if (!pending[sn] || wait_stage(sn)) load_slice(nxt, sn);
        }
        asm volatile("cp.async.commit_group;");
    }
    asm volatile("cp.async.wait_group 0;");
    // drain: every commit still pending (each stage has at most one), bounded, also after a
    // failure, so that no MMA is in flight when the accumulator is read or freed
#pragma unroll
    for (int st = 0; st < S; ++st)
        if (pending[st]) wait_stage(st);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int any_fail = __syncthreads_or(fail);
    if (!any_fail) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                           "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                           "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if constexpr (EPI == 2) {
                // C[col][row]: the lanes' rows are adjacent, so each reduction is coalesced
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < N) atomicAdd(reinterpret_cast<float *>(C) + (size_t)col * M + row, __uint_as_float(r[j]));
                    }
                }
            } else {
                // C[row][col] (bf16): through this warp's 32 x 16 block of shared memory (the stages are
                // free after the drain) so that a store instruction covers two rows of 16
                // adjacent columns instead of 32 rows of one
                float *stg = reinterpret_cast<float *>(smem_raw) + warp * (32 * 17);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float v = __uint_as_float(r[j]);
                    if constexpr (EPI == 0) {
                        const int col = n0 + c0 + j;
                        v += (bias && col < N) ? bias[col] : 0.f;
                        if (relu) v = fmaxf(v, 0.f);
                    }
                    stg[lane * 17 + j] = v;
                }
                __syncwarp();
#pragma unroll
                for (int it = 0; it < 16; ++it) {
                    const int idx = it * 32 + lane, rl = idx >> 4, cl = idx & 15;
                    const int grow = m0 + warp * 32 + rl, col = n0 + c0 + cl;
                    if (grow < M && col < N) {
                        const float v = stg[rl * 17 + cl];
                        reinterpret_cast<bf16 *>(C)[(size_t)grow * N + col] = __float2bfloat16(v);
                    }
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOL));
}

// ----------------------------------------------------------------------------- im2col
// Input of a 3x3 'same' convolution at resolution H x W is the channel concatenation of
// source a (ca channels, stored at H/ua x W/ua, nearest upsampling by ua in {1, 2}) and
// source b (cb channels, H x W; cb may be 0). col[p][(dy*3 + dx) * (ca + cb) + ci].
// One work item = (pixel, tap, 8-channel group); channel counts other than the first layer's
// are multiples of 8, so a group is one 16-byte copy. Indices fit 32 bits (P * 9 * cin < 2^31
// is checked by the host).
__global__ void k_im2col(int B, int H, int W, const bf16 *__restrict__ a, int ca, int ua,
                         const bf16 *__restrict__ b, int cb, bf16 *col) {
    const int cin = ca + cb, K = 9 * cin;
    const int HW = H * W, Ha = H / ua, Wa = W / ua;
    const bool vec = (ca % 8 == 0) && (cb % 8 == 0);
    const int G = vec ? cin / 8 : cin;  // groups per tap
    const unsigned total = (unsigned)B * HW * 9u * (unsigned)G;
    const bf16 zero = __float2bfloat16(0.f);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const unsigned grp = i % (unsigned)G;
        const unsigned pt = i / (unsigned)G;  // pixel * 9 + tap
        const unsigned tap = pt % 9u, p = pt / 9u;
        const int n = (int)(p / (unsigned)HW), rem = (int)(p % (unsigned)HW);
        const int y = rem / W + (int)(tap / 3u) - 1, x = rem % W + (int)(tap % 3u) - 1;
        const bool in = y >= 0 && y < H && x >= 0 && x < W;
        bf16 *dst = col + (size_t)p * K + tap * cin;
        if (vec) {
            const int ci = grp * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (in) {
                const bf16 *src = ci < ca ? a + (((size_t)n * Ha + y / ua) * Wa + x / ua) * ca + ci
                                          : b + (((size_t)n * H + y) * W + x) * cb + (ci - ca);
                v = *reinterpret_cast<const uint4 *>(src);
            }
            *reinterpret_cast<uint4 *>(dst + ci) = v;
        } else {
            const int ci = grp;
            bf16 v = zero;
            if (in) v = ci < ca ? a[(((size_t)n * Ha + y / ua) * Wa + x / ua) * ca + ci]
                                : b[(((size_t)n * H + y) * W + x) * cb + (ci - ca)];
            dst[ci] = v;
        }
    }
}

// Adjoint of k_im2col: from dcol (fp32, [p][K]) form the gradients of sources a and b (fp32,
// same layouts as the forward sources). Gather form: each source element sums the col
// entries that read it, so no atomics are needed. One thread per (source pixel, channel).
__global__ void k_col2im(int B, int H, int W, const float *__restrict__ dcol, float *da, int ca,
                         int ua, float *db, int cb) {
    const int cin = ca + cb, K = 9 * cin;
    const int Ha = H / ua, Wa = W / ua;
    const unsigned na = (unsigned)B * Ha * Wa * ca, nbt = (unsigned)B * H * W * cb;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nbt; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        if (i < na) {
            const int ci = (int)(i % (unsigned)ca);
            const unsigned q = i / (unsigned)ca;
            const int X = (int)(q % (unsigned)Wa), Y = (int)((q / (unsigned)Wa) % (unsigned)Ha);
            const int n = (int)(q / (unsigned)(Wa * Ha));
            for (int sy = 0; sy < ua; ++sy)
                for (int sx = 0; sx < ua; ++sx) {
                    const int y = Y * ua + sy, x = X * ua + sx;  // pixel of the upsampled input
                    for (int tap = 0; tap < 9; ++tap) {
                        const int yo = y - (tap / 3 - 1), xo = x - (tap % 3 - 1);  // output pixel
                        if (yo < 0 || yo >= H || xo < 0 || xo >= W) continue;
                        s += dcol[(((size_t)n * H + yo) * W + xo) * K + tap * cin + ci];
                    }
                }
            da[i] = s;
        } else {
            const unsigned j = i - na;
            const int ci = (int)(j % (unsigned)cb);
            const unsigned q = j / (unsigned)cb;
            const int x = (int)(q % (unsigned)W), y = (int)((q / (unsigned)W) % (unsigned)H);
            const int n = (int)(q / (unsigned)(W * H));
            for (int tap = 0; tap < 9; ++tap) {
                const int yo = y - (tap / 3 - 1), xo = x - (tap % 3 - 1);
                if (yo < 0 || yo >= H || xo < 0 || xo >= W) continue;
                s += dcol[(((size_t)n * H + yo) * W + xo) * K + tap * cin + ca + ci];
            }
            db[j] = s;
        }
    }
}

// out[c][r] = in[r][c] for a bf16 matrix of R rows and C columns (32 x 32 tiles through shared
// memory, coalesced on both sides): the K-major operands of the backward tcgen05 GEMMs.
// Grid: (ceil(R / 32), ceil(C / 32)) (rows, the long side, on x), 256 threads.
__global__ void __launch_bounds__(256)
k_transpose_bf16(const bf16 *__restrict__ in, bf16 *out, int R, int C) {
    __shared__ bf16 t[32][34];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int r = r0 + ty + j, c = c0 + tx;
        if (r < R && c < C) t[ty + j][tx] = in[(size_t)r * C + c];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int c = c0 + ty + j, r = r0 + tx;
        if (r < R && c < C) out[(size_t)c * R + r] = t[tx][ty + j];
    }
}

// ------------------------------------------------------------------- elementwise / small
// dz = dy * (y > 0) rounded to bf16 (the ReLU's backward; y is the post-ReLU output).
__global__ void k_relu_bwd(size_t n, const float *__restrict__ dy, const bf16 *__restrict__ y,
                           int relu, bf16 *dz) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float g = dy[i];
        if (relu && !(__bfloat162float(y[i]) > 0.f)) g = 0.f;
        dz[i] = __float2bfloat16(g);
    }
}

// 2x2 max pooling, NHWC.
__global__ void k_maxpool(int B, int H, int W, int C, const bf16 *__restrict__ in, bf16 *out) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t total = (size_t)B * Ho * Wo * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int x = (int)(q % Wo), y = (int)((q / Wo) % Ho), n = (int)(q / ((size_t)Wo * Ho));
        float m = -3.0e38f;
        for (int s = 0; s < 4; ++s) {
            const float v = __bfloat162float(in[(((size_t)n * H + 2 * y + (s >> 1)) * W + 2 * x + (s & 1)) * C + c]);
            m = fmaxf(m, v);
        }
        out[i] = __float2bfloat16(m);
    }
}

// Backward of 2x2 max pooling: the gradient goes to the first maximal element of each window.
// dinp += routed gradient (dinp already holds the skip-connection gradient).
__global__ void k_maxpool_bwd(int B, int H, int W, int C, const bf16 *__restrict__ in,
                              const float *__restrict__ dout, float *dinp) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t total = (size_t)B * Ho * Wo * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int x = (int)(q % Wo), y = (int)((q / Wo) % Ho), n = (int)(q / ((size_t)Wo * Ho));
        float m = -3.0e38f;
        int arg = 0;
        for (int s = 0; s < 4; ++s) {
            const float v = __bfloat162float(in[(((size_t)n * H + 2 * y + (s >> 1)) * W + 2 * x + (s & 1)) * C + c]);
            if (v > m) { m = v; arg = s; }
        }
        dinp[(((size_t)n * H + 2 * y + (arg >> 1)) * W + 2 * x + (arg & 1)) * C + c] += dout[i];
    }
}

// Head: 1x1 convolution C -> 1 (fp32 out) and its backward.
__global__ void k_head(size_t P, int C, const bf16 *__restrict__ in, const float *__restrict__ w,
                       const float *__restrict__ b, float *out) {
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < C; ++c) s += w[c] * __bfloat162float(in[p * C + c]);
        out[p] = s;
    }
}

// MSE loss L = mean((out - tgt)^2): dout = 2 (out - tgt) / P; partial sums of (out - tgt)^2.
__global__ void k_mse(size_t P, const float *__restrict__ out, const float *__restrict__ tgt,
                      float *dout, double *part) {
    __shared__ double red[32];
    double s = 0.0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const float d = out[p] - tgt[p];
        dout[p] = 2.0f * d / (float)P;
        s += (double)d * (double)d;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Head backward: dW[c] += sum_p dout[p] in[p][c]; db += sum dout; din[p][c] = dout[p] w[c].
__global__ void k_head_bwd(size_t P, int C, const bf16 *__restrict__ in, const float *__restrict__ w,
                           const float *__restrict__ dout, float *dw, float *db, float *din) {
    __shared__ float sw[256];
    __shared__ float sb;
    for (int c = threadIdx.x; c < C; c += blockDim.x) sw[c] = 0.f;
    if (threadIdx.x == 0) sb = 0.f;
    __syncthreads();
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const float g = dout[p];
        atomicAdd(&sb, g);
        for (int c = 0; c < C; ++c) {
            atomicAdd(&sw[c], g * __bfloat162float(in[p * C + c]));
            din[p * C + c] = g * w[c];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&dw[c], sw[c]);
    if (threadIdx.x == 0) atomicAdd(db, sb);
}

// Bias gradient: db[c] += sum_p dz[p][c] (C a multiple of 8). Thread t reads 16 bytes (8
// channels) of rows t / (C / 8) + k (blockDim.x / (C / 8)) of its CTA's row range; the CTA sums
// its threads' partials per channel in shared memory and adds them once. blockDim.x = 256.
__global__ void __launch_bounds__(256) k_bias_grad(size_t P, int C, const bf16 *__restrict__ dz, float *db) {
    __shared__ float part[256 * 8];
    const int nq = C >> 3, rows = blockDim.x / nq;
    const int q = threadIdx.x % nq, r0 = threadIdx.x / nq;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r0 < rows) {
        for (size_t p = (size_t)blockIdx.x * rows + r0; p < P; p += (size_t)gridDim.x * rows) {
            const uint4 v = *reinterpret_cast<const uint4 *>(dz + p * C + (size_t)q * 8);
            const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(e[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) part[threadIdx.x * 8 + j] = acc[j];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int cq = c >> 3, cj = c & 7;
        float s = 0.f;
        for (int r = 0; r < rows; ++r) s += part[(r * nq + cq) * 8 + cj];
        atomicAdd(&db[c], s);
    }
}
// Pack the two network inputs (fp32 planes [B][2][H][W]) into NHWC bf16 [B][H][W][2].
__global__ void k_pack_input(int B, int H, int W, const float *__restrict__ in, bf16 *out) {
    const size_t total = (size_t)B * H * W;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const size_t n = p / ((size_t)H * W), r = p - n * H * W;
        out[2 * p] = __float2bfloat16(in[(n * 2) * H * W + r]);
        out[2 * p + 1] = __float2bfloat16(in[(n * 2 + 1) * H * W + r]);
    }
}

// The warm start's network input, one image straight from the solver's planes (float or
// double [H][W]): NHWC bf16 [H][W][2] = (s0 a, s1 b), the products taken in T.
template <typename T>
__global__ void k_pack_planes(size_t P, const T *__restrict__ a, const T *__restrict__ b, T s0, T s1, bf16 *out) {
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        out[2 * p] = __float2bfloat16((float)(s0 * a[p]));
        out[2 * p + 1] = __float2bfloat16((float)(s1 * b[p]));
    }
}

// Scaled float planes from the solver's planes: out[0] = s0 a, out[1] = s1 b (b may be null:
// one plane), products in T, each plane [P].
template <typename T>
__global__ void k_scale_planes(size_t P, const T *__restrict__ a, const T *__restrict__ b, T s0, T s1, float *out) {
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        out[p] = (float)(s0 * a[p]);
        if (b) out[P + p] = (float)(s1 * b[p]);
    }
}

// The warm start itself: x0 = max(s out, 0) in the solver's type.
template <typename T>
__global__ void k_x0_from_output(size_t P, const float *__restrict__ out, T s, T *x0) {
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const T v = s * (T)out[p];
        x0[p] = v > (T)0 ? v : (T)0;
    }
}

// Adam on fp32 masters; refresh the bf16 copies. step >= 1.
__global__ void k_adam(size_t n, float *w, const float *__restrict__ g, float *m, float *v, bf16 *wb,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(size_t n, const float *__restrict__ in, bf16 *out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(in[i]);
}

}  // namespace ivis
