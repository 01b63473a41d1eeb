// unet.cu -- the learned warm start: a 4-level U-Net that maps [dirty image, beam-weight map]
// to an initial sky for the solver (see include/ivis.h, ivis_unet_*). Training and inference
// run in this library's own kernels (kernels_unet.cuh).
//
// Architecture (base width c = 32): per level two 3x3 convolutions with ReLU; encoder widths
// c, 2c, 4c, 8c at H, H/2, H/4, H/8 with 2x2 max pooling between levels; decoder: nearest 2x
// upsampling, concatenation with the encoder output of the same level, two 3x3 convolutions
// with ReLU (widths 4c, 2c, c); a 1x1 head to one output plane. Loss: mean squared error.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ivis.h"
#include "kernels_unet.cuh"

using namespace ivis;

namespace {

struct ConvSpec {
    int src_a, ca, ua;  // tensor id, channels, upsampling of source a
    int src_b, cb;      // tensor id and channels of source b (concatenated), or -1 / 0
    int cout, level;    // output channels, resolution level (H >> level)
    int out;            // output tensor id
    size_t w_off, b_off;
};

thread_local std::string g_unet_err;

}  // namespace

struct ivis_unet_s {
    int c = 32, max_batch = 0, max_hw = 0;
    cudaStream_t stream = nullptr;
    std::vector<ConvSpec> convs;
    int ntensor = 0;
    std::vector<int> tch, tlev;          // channels and level of each activation tensor
    size_t nparam = 0, head_w = 0, head_b = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wb = nullptr;
    std::vector<bf16 *> act;             // activations (bf16 NHWC)
    std::vector<float *> dact;           // their gradients (fp32)
    bf16 *col = nullptr, *dz = nullptr;
    bf16 *colT = nullptr, *dzT = nullptr;  // K-major operands of the tcgen05 parameter gradients
    float *dcol = nullptr, *out = nullptr, *dout = nullptr, *tgt = nullptr;
    double *part = nullptr, *part_h = nullptr;
    size_t col_cap = 0, dz_cap = 0;
    long long step = 0;
    bool use_tc = true;   // convolutions and their gradients on tcgen05 (else mma.sync)
    int *tc_err = nullptr;
    std::string err;
};

namespace {

ivis_status ufail(ivis_unet_s *u, ivis_status s, const std::string &msg) {
    if (u) u->err = msg;
    g_unet_err = msg;
    return s;
}

#define UCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return ufail(u, IVIS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// tensor ids
enum { T_IN = 0, T_A0, T_A1, T_P0, T_A2, T_A3, T_P1, T_A4, T_A5, T_P2, T_A6, T_A7, T_A8, T_A9,
       T_A10, T_A11, T_A12, T_A13, T_COUNT };

void build_net(ivis_unet_s *u) {
    const int c = u->c;
    u->ntensor = T_COUNT;
    u->tch.assign(T_COUNT, 0);
    u->tlev.assign(T_COUNT, 0);
    auto T = [&](int id, int ch, int lev) { u->tch[id] = ch; u->tlev[id] = lev; };
    T(T_IN, 2, 0);
    T(T_A0, c, 0); T(T_A1, c, 0); T(T_P0, c, 1);
    T(T_A2, 2 * c, 1); T(T_A3, 2 * c, 1); T(T_P1, 2 * c, 2);
    T(T_A4, 4 * c, 2); T(T_A5, 4 * c, 2); T(T_P2, 4 * c, 3);
    T(T_A6, 8 * c, 3); T(T_A7, 8 * c, 3);
    T(T_A8, 4 * c, 2); T(T_A9, 4 * c, 2);
    T(T_A10, 2 * c, 1); T(T_A11, 2 * c, 1);
    T(T_A12, c, 0); T(T_A13, c, 0);
    auto C = [&](int a, int ua, int b, int out) {
        ConvSpec s{};
        s.src_a = a; s.ca = u->tch[a]; s.ua = ua;
        s.src_b = b; s.cb = b >= 0 ? u->tch[b] : 0;
        s.cout = u->tch[out]; s.level = u->tlev[out]; s.out = out;
        u->convs.push_back(s);
    };
    C(T_IN, 1, -1, T_A0); C(T_A0, 1, -1, T_A1);
    C(T_P0, 1, -1, T_A2); C(T_A2, 1, -1, T_A3);
    C(T_P1, 1, -1, T_A4); C(T_A4, 1, -1, T_A5);
    C(T_P2, 1, -1, T_A6); C(T_A6, 1, -1, T_A7);
    C(T_A7, 2, T_A5, T_A8); C(T_A8, 1, -1, T_A9);
    C(T_A9, 2, T_A3, T_A10); C(T_A10, 1, -1, T_A11);
    C(T_A11, 2, T_A1, T_A12); C(T_A12, 1, -1, T_A13);
    size_t off = 0;
    for (auto &s : u->convs) {
        s.w_off = off;
        off += (size_t)s.cout * 9 * (s.ca + s.cb);
        s.b_off = off;
        off += s.cout;
    }
    u->head_w = off;
    off += c;
    u->head_b = off;
    off += 1;
    u->nparam = off;
}

unsigned nblk(size_t n, int t = 256) { return (unsigned)std::min<size_t>((n + t - 1) / t, 148 * 32); }

ivis_status ensure_scratch(ivis_unet_s *u, size_t col_elems, size_t dz_elems) {
    if (col_elems > u->col_cap) {
        if (u->col) cudaFree(u->col);
        if (u->dcol) cudaFree(u->dcol);
        if (u->colT) cudaFree(u->colT);
        u->col = nullptr; u->dcol = nullptr; u->colT = nullptr;
        if (cudaMalloc(&u->col, col_elems * sizeof(bf16)) != cudaSuccess ||
            cudaMalloc(&u->dcol, col_elems * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&u->colT, col_elems * sizeof(bf16)) != cudaSuccess) {
            cudaGetLastError();
            u->col_cap = 0;
            return ufail(u, IVIS_ERR_OOM, "U-Net scratch allocation failed");
        }
        u->col_cap = col_elems;
    }
    if (dz_elems > u->dz_cap) {
        if (u->dz) cudaFree(u->dz);
        if (u->dzT) cudaFree(u->dzT);
        u->dz = nullptr; u->dzT = nullptr;
        if (cudaMalloc(&u->dz, dz_elems * sizeof(bf16)) != cudaSuccess ||
            cudaMalloc(&u->dzT, dz_elems * sizeof(bf16)) != cudaSuccess) {
            cudaGetLastError();
            u->dz_cap = 0;
            return ufail(u, IVIS_ERR_OOM, "U-Net scratch allocation failed");
        }
        u->dz_cap = dz_elems;
    }
    return IVIS_OK;
}

template <int BN, bool IMPLICIT, int EPI>
void gemm_tc_launch(cudaStream_t st, int M, int N, int K, int kchunk, const bf16 *A, const bf16 *B, void *C,
                    const float *bias, int relu, int *err, ConvGeom cg) {
    constexpr int NCOL = BN < 32 ? 32 : BN;
    const size_t need = (size_t)tc_stages<BN>::value * (TC_BM + BN) * TC_BK * sizeof(bf16) + 64;
    // keep the CTAs resident on one SM within its 512 TMEM columns
    const int allowed = 512 / NCOL;
    const size_t smem = std::max(need, (size_t)(228 * 1024) / (allowed + 1) + 1024);
    cudaFuncSetAttribute(k_gemm_tc<BN, IMPLICIT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 g((M + TC_BM - 1) / TC_BM, (N + BN - 1) / BN, (K + kchunk - 1) / kchunk);
    k_gemm_tc<BN, IMPLICIT, EPI><<<g, 128, smem, st>>>(M, N, K, kchunk, A, B, C, bias, relu, err, cg);
}

// cg.a == nullptr: explicit A (an im2col matrix); otherwise A is gathered from cg.
// kchunk: split of K over gridDim.z (rounded up to a multiple of TC_BK; EPI 2 only), 0 = none.
template <bool IMPLICIT, int EPI>
void gemm_tc_n(cudaStream_t st, int M, int N, int K, int kchunk, const bf16 *A, const bf16 *B, void *C,
               const float *bias, int relu, int *err, ConvGeom cg) {
    kchunk = kchunk > 0 ? (kchunk + TC_BK - 1) / TC_BK * TC_BK : K;
    if (N <= 16) gemm_tc_launch<16, IMPLICIT, EPI>(st, M, N, K, kchunk, A, B, C, bias, relu, err, cg);
    else if (N <= 32) gemm_tc_launch<32, IMPLICIT, EPI>(st, M, N, K, kchunk, A, B, C, bias, relu, err, cg);
    else if (N <= 64) gemm_tc_launch<64, IMPLICIT, EPI>(st, M, N, K, kchunk, A, B, C, bias, relu, err, cg);
    else if (N <= 128) gemm_tc_launch<128, IMPLICIT, EPI>(st, M, N, K, kchunk, A, B, C, bias, relu, err, cg);
    else gemm_tc_launch<256, IMPLICIT, EPI>(st, M, N, K, kchunk, A, B, C, bias, relu, err, cg);
}

void gemm_tc(cudaStream_t st, int M, int N, int K, const bf16 *A, const bf16 *B, bf16 *C,
             const float *bias, int relu, int *err, ConvGeom cg = ConvGeom{}) {
    if (cg.a) gemm_tc_n<true, 0>(st, M, N, K, 0, A, B, C, bias, relu, err, cg);
    else gemm_tc_n<false, 0>(st, M, N, K, 0, A, B, C, bias, relu, err, cg);
}

// Parameter-gradient GEMM on tcgen05: C fp32 [N][M] += A B^T with K split into chunks of kchunk
// (EPI 2); both operands K-major bf16.
void gemm_tc_wgrad(cudaStream_t st, int M, int N, int K, int kchunk, const bf16 *A, const bf16 *B, float *C,
                   int *err) {
    gemm_tc_n<false, 2>(st, M, N, K, kchunk, A, B, C, nullptr, 0, err, ConvGeom{});
}

void gemm(cudaStream_t st, int ta, int tb, int epi, int M, int N, int K, const bf16 *A, const bf16 *B,
          void *Cm, const float *bias, int relu, int splitk_chunk = 0) {
    int kchunk = splitk_chunk > 0 ? splitk_chunk : K;
    kchunk = (kchunk + GB_K - 1) / GB_K * GB_K;
    dim3 g((M + GB_M - 1) / GB_M, (N + GB_N - 1) / GB_N, (K + kchunk - 1) / kchunk);
    if (ta == 0 && tb == 1 && epi == 0) k_gemm_bf16<0, 1, 0><<<g, 256, 0, st>>>(M, N, K, kchunk, A, B, Cm, bias, relu);
    else if (ta == 1 && tb == 0 && epi == 2) k_gemm_bf16<1, 0, 2><<<g, 256, 0, st>>>(M, N, K, kchunk, A, B, Cm, bias, relu);
    else if (ta == 0 && tb == 0 && epi == 1) k_gemm_bf16<0, 0, 1><<<g, 256, 0, st>>>(M, N, K, kchunk, A, B, Cm, bias, relu);
}

ivis_status check_shape(ivis_unet_s *u, int B, int H, int W) {
    if (B < 1 || B > u->max_batch) return ufail(u, IVIS_ERR_ARG, "batch outside [1, max_batch]");
    if (H < 8 || W < 8 || H % 8 || W % 8) return ufail(u, IVIS_ERR_ARG, "H and W must be multiples of 8");
    if ((size_t)H * W > (size_t)u->max_hw) return ufail(u, IVIS_ERR_ARG, "H*W above max_hw");
    // 32-bit work-item indices of the im2col / col2im kernels: P * 9 * cin < 2^31 per layer
    for (auto &c : u->convs)
        if ((size_t)B * (H >> c.level) * (W >> c.level) * 9 * (c.ca + c.cb) >= (size_t)1 << 31)
            return ufail(u, IVIS_ERR_ARG, "batch x image too large for one call");
    return IVIS_OK;
}

// in_dev == nullptr: the caller has packed the input tensor already.
ivis_status forward_impl(ivis_unet_s *u, const float *in_dev, int B, int H, int W) {
    cudaStream_t st = u->stream;
    const size_t P0 = (size_t)B * H * W;
    if (in_dev) k_pack_input<<<nblk(P0), 256, 0, st>>>(B, H, W, in_dev, u->act[T_IN]);
    for (size_t li = 0; li < u->convs.size(); ++li) {
        const ConvSpec &s = u->convs[li];
        const int h = H >> s.level, w = W >> s.level;
        const size_t P = (size_t)B * h * w;
        const int K = 9 * (s.ca + s.cb);
        const bf16 *srcb = s.src_b >= 0 ? u->act[s.src_b] : nullptr;
        if (u->use_tc && s.ca % 8 == 0 && s.cb % 8 == 0 && h < 32768 && w < 32768) {
            // implicit GEMM: the 3x3 gather happens in the operand copies
            gemm_tc(st, (int)P, s.cout, K, nullptr, u->wb + s.w_off, u->act[s.out], u->w + s.b_off, 1, u->tc_err,
                    ConvGeom{u->act[s.src_a], srcb, s.ca, s.ua, s.cb, h, w});
        } else {
            k_im2col<<<nblk(P * K), 256, 0, st>>>(B, h, w, u->act[s.src_a], s.ca, s.ua, srcb, s.cb, u->col);
            if (u->use_tc)
                gemm_tc(st, (int)P, s.cout, K, u->col, u->wb + s.w_off, u->act[s.out], u->w + s.b_off, 1, u->tc_err);
            else
                gemm(st, 0, 1, 0, (int)P, s.cout, K, u->col, u->wb + s.w_off, u->act[s.out], u->w + s.b_off, 1);
        }
        // pooling after the second convolution of each encoder level
        if (s.out == T_A1 || s.out == T_A3 || s.out == T_A5) {
            const int pid = s.out == T_A1 ? T_P0 : (s.out == T_A3 ? T_P1 : T_P2);
            k_maxpool<<<nblk(P / 4 * s.cout), 256, 0, st>>>(B, h, w, s.cout, u->act[s.out], u->act[pid]);
        }
    }
    k_head<<<nblk(P0), 256, 0, st>>>(P0, u->c, u->act[T_A13], u->w + u->head_w, u->w + u->head_b, u->out);
    UCK(cudaGetLastError());
    if (u->use_tc) {
        int herr = 0;
        UCK(cudaMemcpyAsync(&herr, u->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        UCK(cudaStreamSynchronize(st));
        if (herr) return ufail(u, IVIS_ERR_TIMEOUT, "tensor-core GEMM: completion wait timed out");
    }
    return IVIS_OK;
}

}  // namespace

extern "C" {

ivis_status ivis_unet_create(int base_channels, int max_batch, int max_hw, void *stream, ivis_unet_t *out) {
    if (!out) return ufail(nullptr, IVIS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (base_channels < 8 || base_channels > 64 || base_channels % 8)
        return ufail(nullptr, IVIS_ERR_ARG, "base_channels must be a multiple of 8 in [8, 64]");
    if (max_batch < 1 || max_hw < 64) return ufail(nullptr, IVIS_ERR_ARG, "max_batch >= 1 and max_hw >= 64 required");
    ivis_unet_s *u = new (std::nothrow) ivis_unet_s();
    if (!u) return ufail(nullptr, IVIS_ERR_OOM, "host allocation failed");
    u->c = base_channels;
    u->max_batch = max_batch;
    u->max_hw = max_hw;
    u->stream = (cudaStream_t)stream;
    build_net(u);
    bool ok = cudaMalloc(&u->w, u->nparam * 4) == cudaSuccess && cudaMalloc(&u->g, u->nparam * 4) == cudaSuccess &&
              cudaMalloc(&u->m, u->nparam * 4) == cudaSuccess && cudaMalloc(&u->v, u->nparam * 4) == cudaSuccess &&
              cudaMalloc(&u->wb, u->nparam * 2) == cudaSuccess;
    u->act.assign(u->ntensor, nullptr);
    u->dact.assign(u->ntensor, nullptr);
    for (int t = 0; t < u->ntensor && ok; ++t) {
        const size_t n = (size_t)max_batch * (max_hw >> (2 * u->tlev[t])) * u->tch[t];
        ok = cudaMalloc(&u->act[t], n * sizeof(bf16)) == cudaSuccess &&
             cudaMalloc(&u->dact[t], n * sizeof(float)) == cudaSuccess;
    }
    const size_t P0 = (size_t)max_batch * max_hw;
    ok = ok && cudaMalloc(&u->out, P0 * 4) == cudaSuccess && cudaMalloc(&u->dout, P0 * 4) == cudaSuccess &&
         cudaMalloc(&u->tgt, P0 * 4) == cudaSuccess && cudaMalloc(&u->part, 148 * 32 * sizeof(double)) == cudaSuccess &&
         cudaMallocHost(&u->part_h, 148 * 32 * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&u->tc_err, sizeof(int)) == cudaSuccess;
    if (ok) cudaMemset(u->tc_err, 0, sizeof(int));
    if (ok) {
        cudaMemset(u->w, 0, u->nparam * 4);
        cudaMemset(u->g, 0, u->nparam * 4);
        cudaMemset(u->m, 0, u->nparam * 4);
        cudaMemset(u->v, 0, u->nparam * 4);
        cudaMemset(u->wb, 0, u->nparam * 2);
    }
    if (!ok) {
        cudaGetLastError();
        ivis_unet_destroy(u);
        return ufail(nullptr, IVIS_ERR_OOM, "U-Net device allocation failed");
    }
    *out = u;
    return IVIS_OK;
}

ivis_status ivis_unet_num_params(ivis_unet_t u, int64_t *n) {
    if (!u || !n) return ufail(u, IVIS_ERR_ARG, "null pointer");
    *n = (int64_t)u->nparam;
    return IVIS_OK;
}

ivis_status ivis_unet_set_params(ivis_unet_t u, const float *host_params) {
    if (!u || !host_params) return ufail(u, IVIS_ERR_ARG, "null pointer");
    UCK(cudaMemcpyAsync(u->w, host_params, u->nparam * 4, cudaMemcpyHostToDevice, u->stream));
    k_to_bf16<<<nblk(u->nparam), 256, 0, u->stream>>>(u->nparam, u->w, u->wb);
    UCK(cudaMemsetAsync(u->m, 0, u->nparam * 4, u->stream));
    UCK(cudaMemsetAsync(u->v, 0, u->nparam * 4, u->stream));
    UCK(cudaStreamSynchronize(u->stream));
    u->step = 0;
    return IVIS_OK;
}

ivis_status ivis_unet_get_params(ivis_unet_t u, float *host_params) {
    if (!u || !host_params) return ufail(u, IVIS_ERR_ARG, "null pointer");
    UCK(cudaMemcpyAsync(host_params, u->w, u->nparam * 4, cudaMemcpyDeviceToHost, u->stream));
    UCK(cudaStreamSynchronize(u->stream));
    return IVIS_OK;
}

ivis_status ivis_unet_get_grads(ivis_unet_t u, float *host_grads) {
    if (!u || !host_grads) return ufail(u, IVIS_ERR_ARG, "null pointer");
    UCK(cudaMemcpyAsync(host_grads, u->g, u->nparam * 4, cudaMemcpyDeviceToHost, u->stream));
    UCK(cudaStreamSynchronize(u->stream));
    return IVIS_OK;
}

ivis_status ivis_unet_forward(ivis_unet_t u, const float *in_dev, float *out_dev, int B, int H, int W) {
    if (!u || !in_dev || !out_dev) return ufail(u, IVIS_ERR_ARG, "null pointer");
    ivis_status s = check_shape(u, B, H, W);
    if (s) return s;
    size_t colmax = 0;
    for (auto &c : u->convs) colmax = std::max(colmax, (size_t)B * (H >> c.level) * (W >> c.level) * 9 * (c.ca + c.cb));
    if ((s = ensure_scratch(u, colmax, 1))) return s;
    if ((s = forward_impl(u, in_dev, B, H, W))) return s;
    UCK(cudaMemcpyAsync(out_dev, u->out, (size_t)B * H * W * 4, cudaMemcpyDeviceToDevice, u->stream));
    UCK(cudaStreamSynchronize(u->stream));
    return IVIS_OK;
}

ivis_status ivis_unet_warm_start(ivis_unet_t u, const void *dirty_dev, const void *beamw_dev, int fp64, int H,
                                 int W, double s0, double s1, double s_out, void *x0_dev) {
    if (!u || !dirty_dev || !beamw_dev || !x0_dev) return ufail(u, IVIS_ERR_ARG, "null pointer");
    if (!std::isfinite(s0) || !std::isfinite(s1) || !std::isfinite(s_out))
        return ufail(u, IVIS_ERR_ARG, "scales must be finite");
    ivis_status s = check_shape(u, 1, H, W);
    if (s) return s;
    size_t colmax = 0;
    for (auto &c : u->convs) colmax = std::max(colmax, (size_t)(H >> c.level) * (W >> c.level) * 9 * (c.ca + c.cb));
    if ((s = ensure_scratch(u, colmax, 1))) return s;
    cudaStream_t st = u->stream;
    const size_t P = (size_t)H * W;
    if (fp64)
        k_pack_planes<double><<<nblk(P), 256, 0, st>>>(P, (const double *)dirty_dev, (const double *)beamw_dev, s0,
                                                       s1, u->act[T_IN]);
    else
        k_pack_planes<float><<<nblk(P), 256, 0, st>>>(P, (const float *)dirty_dev, (const float *)beamw_dev,
                                                      (float)s0, (float)s1, u->act[T_IN]);
    if ((s = forward_impl(u, nullptr, 1, H, W))) return s;
    if (fp64) k_x0_from_output<double><<<nblk(P), 256, 0, st>>>(P, u->out, s_out, (double *)x0_dev);
    else k_x0_from_output<float><<<nblk(P), 256, 0, st>>>(P, u->out, (float)s_out, (float *)x0_dev);
    UCK(cudaGetLastError());
    UCK(cudaStreamSynchronize(st));
    return IVIS_OK;
}

ivis_status ivis_unet_planes(const void *a_dev, const void *b_dev, int fp64, int64_t npix, double sa, double sb,
                             float *out_dev, void *stream) {
    if (!a_dev || !out_dev) return ufail(nullptr, IVIS_ERR_ARG, "null pointer");
    if (npix < 0) return ufail(nullptr, IVIS_ERR_ARG, "negative pixel count");
    if (!std::isfinite(sa) || !std::isfinite(sb)) return ufail(nullptr, IVIS_ERR_ARG, "scales must be finite");
    if (npix == 0) return IVIS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = (size_t)npix;
    if (fp64)
        k_scale_planes<double><<<nblk(P), 256, 0, st>>>(P, (const double *)a_dev, (const double *)b_dev, sa, sb, out_dev);
    else
        k_scale_planes<float><<<nblk(P), 256, 0, st>>>(P, (const float *)a_dev, (const float *)b_dev, (float)sa,
                                                       (float)sb, out_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ufail(nullptr, IVIS_ERR_CUDA, std::string("unet planes: ") + cudaGetErrorString(e));
    return IVIS_OK;
}

ivis_status ivis_unet_backward(ivis_unet_t u, const float *in_dev, const float *tgt_dev, int B, int H,
                               int W, double *loss_out) {
    if (!u || !in_dev || !tgt_dev) return ufail(u, IVIS_ERR_ARG, "null pointer");
    ivis_status s = check_shape(u, B, H, W);
    if (s) return s;
    cudaStream_t st = u->stream;
    size_t colmax = 0, dzmax = 0;
    for (auto &c : u->convs) {
        const size_t P = (size_t)B * (H >> c.level) * (W >> c.level);
        colmax = std::max(colmax, P * 9 * (c.ca + c.cb));
        dzmax = std::max(dzmax, P * c.cout);
    }
    if ((s = ensure_scratch(u, colmax, dzmax))) return s;
    if ((s = forward_impl(u, in_dev, B, H, W))) return s;
    const size_t P0 = (size_t)B * H * W;
    UCK(cudaMemsetAsync(u->g, 0, u->nparam * 4, st));
    const unsigned nb_mse = nblk(P0);
    k_mse<<<nb_mse, 256, 0, st>>>(P0, u->out, tgt_dev, u->dout, u->part);
    k_head_bwd<<<nblk(P0), 256, 0, st>>>(P0, u->c, u->act[T_A13], u->w + u->head_w, u->dout,
                                         u->g + u->head_w, u->g + u->head_b, u->dact[T_A13]);
    for (int li = (int)u->convs.size() - 1; li >= 0; --li) {
        const ConvSpec &c = u->convs[li];
        const int h = H >> c.level, w = W >> c.level;
        const size_t P = (size_t)B * h * w;
        const int K = 9 * (c.ca + c.cb);
        k_relu_bwd<<<nblk(P * c.cout), 256, 0, st>>>(P * c.cout, u->dact[c.out], u->act[c.out], 1, u->dz);
        k_im2col<<<nblk(P * K), 256, 0, st>>>(B, h, w, u->act[c.src_a], c.ca, c.ua,
                                               c.src_b >= 0 ? u->act[c.src_b] : nullptr, c.cb, u->col);
        // dW += dz^T col (split over pixels), db += sum dz, dcol = dz W
        if (u->use_tc) {
            // tcgen05 wants both operands K-major: dW^T [K][cout] += col^T (dz^T)^T over the
            // pixels (split in chunks of 8192), from transposed copies of col and dz
            k_transpose_bf16<<<dim3((unsigned)((P + 31) / 32), (c.cout + 31) / 32), 256, 0, st>>>(u->dz, u->dzT,
                                                                                               (int)P, c.cout);
            k_transpose_bf16<<<dim3((unsigned)((P + 31) / 32), (K + 31) / 32), 256, 0, st>>>(u->col, u->colT,
                                                                                          (int)P, K);
            gemm_tc_wgrad(st, K, c.cout, (int)P, 8192, u->colT, u->dzT, u->g + c.w_off, u->tc_err);
        } else {
            gemm(st, 1, 0, 2, c.cout, K, (int)P, u->dz, u->col, u->g + c.w_off, nullptr, 0, 8192);
        }
        const size_t brows = 256 / (c.cout / 8);  // rows per CTA pass of k_bias_grad
        k_bias_grad<<<(unsigned)std::min<size_t>((P + brows - 1) / brows, 148 * 4), 256, 0, st>>>(P, c.cout, u->dz,
                                                                                           u->g + c.b_off);
        if (li == 0) continue;  // no gradient needed for the network input
        // dcol = dz W on mma.sync in both modes: its K is the output channels (32-256), one to
        // four 64-deep slices per tcgen05 tile, where tile set-up and the fp32 epilogue made
        // the tcgen05 version slower (3.98 ms against 2.94 ms per backward, batch 8 x 256^2)
        gemm(st, 0, 0, 1, (int)P, K, c.cout, u->dz, u->wb + c.w_off, u->dcol, nullptr, 0);
        const int ha = h / c.ua, wa = w / c.ua;
        const size_t nsrc = (size_t)B * ha * wa * c.ca + (c.src_b >= 0 ? P * c.cb : 0);
        k_col2im<<<nblk(nsrc), 256, 0, st>>>(B, h, w, u->dcol, u->dact[c.src_a], c.ca, c.ua,
                                             c.src_b >= 0 ? u->dact[c.src_b] : nullptr, c.cb);
        // the pooled tensor's gradient goes back into its pooling source, which already holds
        // the gradient from the decoder's skip connection (that layer ran earlier in reverse)
        if (c.src_a == T_P0 || c.src_a == T_P1 || c.src_a == T_P2) {
            const int pre = c.src_a == T_P0 ? T_A1 : (c.src_a == T_P1 ? T_A3 : T_A5);
            const int hp = h * 2, wp = w * 2;
            k_maxpool_bwd<<<nblk((size_t)B * h * w * c.ca), 256, 0, st>>>(B, hp, wp, c.ca, u->act[pre],
                                                                          u->dact[c.src_a], u->dact[pre]);
        }
    }
    UCK(cudaGetLastError());
    UCK(cudaMemcpyAsync(u->part_h, u->part, nb_mse * sizeof(double), cudaMemcpyDeviceToHost, st));
    int herr = 0;
    if (u->use_tc) UCK(cudaMemcpyAsync(&herr, u->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    UCK(cudaStreamSynchronize(st));
    if (herr) return ufail(u, IVIS_ERR_TIMEOUT, "tensor-core GEMM: completion wait timed out");
    if (loss_out) {
        double sum = 0.0;
        for (unsigned i = 0; i < nb_mse; ++i) sum += u->part_h[i];
        *loss_out = sum / (double)P0;
    }
    return IVIS_OK;
}

ivis_status ivis_unet_adam_step(ivis_unet_t u, float lr, float beta1, float beta2, float eps) {
    if (!u) return ufail(nullptr, IVIS_ERR_ARG, "null pointer");
    u->step++;
    const float c1 = 1.f - std::pow(beta1, (float)u->step), c2 = 1.f - std::pow(beta2, (float)u->step);
    k_adam<<<nblk(u->nparam), 256, 0, u->stream>>>(u->nparam, u->w, u->g, u->m, u->v, u->wb, lr, beta1,
                                                    beta2, eps, c1, c2);
    UCK(cudaGetLastError());
    UCK(cudaStreamSynchronize(u->stream));
    return IVIS_OK;
}

ivis_status ivis_unet_destroy(ivis_unet_t u) {
    if (!u) return IVIS_OK;
    if (u->stream) cudaStreamSynchronize(u->stream);
    void *ptrs[] = {u->w, u->g, u->m, u->v, u->wb, u->col, u->colT, u->dz, u->dzT, u->dcol, u->out,
                    u->dout, u->tgt, u->part, u->tc_err};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (auto q : u->act) if (q) cudaFree(q);
    for (auto q : u->dact) if (q) cudaFree(q);
    if (u->part_h) cudaFreeHost(u->part_h);
    delete u;
    return IVIS_OK;
}

ivis_status ivis_unet_use_tcgen05(ivis_unet_t u, int enable) {
    if (!u) return ufail(nullptr, IVIS_ERR_ARG, "null pointer");
    u->use_tc = enable != 0;
    return IVIS_OK;
}

const char *ivis_unet_last_error(ivis_unet_t u) { return u ? u->err.c_str() : g_unet_err.c_str(); }

}  // extern "C"
