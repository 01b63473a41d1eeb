// ivis.cu -- plan object and C ABI of the engine (see include/ivis.h).
//
// A plan owns every device buffer of one imaging problem: the pointing beams, the
// visibilities of every (pointing, channel) pair converted to fine-grid coordinates and
// sorted by grid tile, the oversampled grids of all pairs, the image-side buffers and the
// FP64 partial sums. One evaluation of Q_tot and its gradient is a fixed sequence of kernel
// launches; it is captured once into a CUDA graph and replayed, so the host issues one graph
// launch per evaluation and reads back one FP64 cost.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ivis.h"
#include "kernels_image.cuh"
#include "kernels_nufft.cuh"
#include "kernels_packed.cuh"
#include "kernels_solver.cuh"
#include "kernels_feather.cuh"
#include "kernels_sdconv.cuh"
#include "kernels_toeplitz.cuh"
#include "kernels_wstack.cuh"
#include "kernels_grid.cuh"
#include "kernels_gridtc.cuh"

using namespace ivis;

namespace {

thread_local std::string g_plan_error;

struct PairHost {
    bool set = false;
    int m = 0;
    void *coord = nullptr, *vis = nullptr, *w = nullptr;
    int *orig = nullptr;
    std::vector<int> tile_count;  // per sort bin of the fine grid, in sort order
    std::vector<int> block_start; // first sorted visibility of each 8 x 8-cell block (sort order)
    // Toeplitz form (toeplitz = 1): spectrum of Re H [kx][ky], window b [nb][nb], constant C
    void *that = nullptr, *bwin = nullptr;
    double qconst = 0.0;
    // w-stacking (wterm = 1): W entries per visibility, sorted by (plane, tile, cell)
    int nplane = 0;
    double w0 = 0.0;                       // plane k sits at w0 + k dw
    std::vector<int> plane_start;          // first sorted entry of each plane (nplane + 1)
    std::vector<int> plane_tile_count;     // [nplane][ntiles], bins in sort order
    void *e_coord = nullptr, *e_val = nullptr, *e_w = nullptr;
    int *e_orig = nullptr, *e_pos = nullptr;
    void *v_vis = nullptr, *v_w = nullptr, *v_phase = nullptr, *v_wk = nullptr;  // caller order
};

struct Stage {
    const char *name;
    cudaEvent_t b, e;  // recorded by event nodes of the profiled graph
    double ms;         // accumulated milliseconds
};
constexpr int MAX_STAGES = 16;

}  // namespace

struct ivis_plan_s {
    ivis_config cfg{};
    cudaStream_t user_stream = nullptr;      // the caller's stream (may be the legacy default)
    cudaStream_t stream = nullptr, side = nullptr;  // the plan's own capturable streams
    cudaStream_t side2 = nullptr;                     // clearing of G beside the adjoint row pass
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_in = nullptr;
    cudaEvent_t ev_cfork = nullptr, ev_cjoin = nullptr;
    bool fp64 = true;
    size_t rsz = 8;  // sizeof(real)
    int nf = 0, lognf = 0, W = 0;
    double beta = 0.0;
    int tile = 32, ntx = 0, ntiles = 0;  // sort bins (32 x 32 cells) of the fine grid
    int gtile = 32;                      // tile edge of the k_grid_pass work list (32 or 64)
    int xtile = 32, item_len = 32;       // item work list: tile edge, visibilities per item
    int xkern = 1;                       // item pass: 1 scalar (k_grid_cg), 2 tensor-core (k_grid_tc)
    int f_half = 0;  // the last forward pass wrote rows 0 .. nf/2 of F only (packed, real windows)
    int logc_cols = 0;  // log2 columns per CTA in the column FFT passes
    int clear_blocks = 8 * 148;  // CTAs of the grid-stride clearing kernel (8 per SM)
    int chunk_cap = 1024;  // max visibilities per grid-pass chunk
    std::string tuned;     // autotuner decision (for reporting)
    std::vector<double> dinv_h;
    void *dinv_d = nullptr, *tw_d = nullptr, *beams_d = nullptr;
    float *kpoly_d = nullptr;  // per-tap kernel polynomials (FP32 path)
    std::vector<int> cx, cy;
    std::vector<char> pset;
    std::vector<int> pgrid;       // 1: pointing k re-projects through its interpolation grid
    void *grids_d = nullptr;      // float2 [npoint][nb][nb] sampling locations (X, Y)
    std::vector<PairHost> pairs;  // index chan * npoint + k
    // single dish
    std::vector<char> sdset;
    std::vector<double> sig_sd, fwhm_sd;
    void *tsd_d = nullptr;
    // prepared state
    bool prepared = false;
    int nslot = 0;
    std::vector<int> slot_pair;            // slot -> pair index
    std::vector<const int *> slot_tc;      // slot -> per-bin visibility (entry) counts
    std::vector<int> slot_m;               // slot -> visibilities (entries)
    std::vector<int> chunk_first;          // slot -> first chunk (size nslot + 1)
    int nchunk = 0;
    std::vector<const int *> slot_bs;      // slot -> per-block visibility starts (k_grid_cg)
    std::vector<int> xchunk_first;         // slot -> first k_grid_cg chunk (size nslot + 1)
    int nxchunk = 0;
    Chunk *xchunks_d = nullptr;            // k_grid_cg chunks: slot, tile, items [begin, end)
    Item *items_d = nullptr;
    PairInfo *pinfo_d = nullptr;
    void *pdata_d = nullptr;
    Chunk *chunks_d = nullptr;
    int *chan_start_d = nullptr, *chan_list_d = nullptr;
    int Rsd = 0;
    void *taps_d = nullptr;
    // dish-beam convolution by line DFTs of period sd_N >= n + R (0: direct taps)
    int sd_N = 0, sd_logN = 0, sd_logc = 0;
    void *sd_spec_d = nullptr, *sd_tw_d = nullptr;
    double *inv_sig2_d = nullptr;
    void *rowbuf = nullptr, *F = nullptr, *G = nullptr, *contrib = nullptr;
    void *x = nullptr, *g = nullptr, *tmp1 = nullptr, *tmp2 = nullptr, *gradK = nullptr;
    double *jpart = nullptr, *kpart = nullptr, *rpart = nullptr, *cost_d = nullptr;
    double *cost_h = nullptr;  // pinned
    int nkpart = 0, nrpart = 0;
    // Toeplitz form
    ivis_plan_s *toep_sub = nullptr;  // 2nb-window plan that computes T and b at set_vis
    void *wbeam_d = nullptr;          // [npoint][nb][nb] beam x dinv[p] dinv[q] (packed passes)
    void **that_ptr_d = nullptr, **bwin_ptr_d = nullptr;  // per slot
    double *qconst_d = nullptr;       // per slot
    int njpart = 0;                   // FP64 data-term partials summed by k_finalize
    // w-stacking
    double w_xc = 0.0, w_dw = 0.0;         // centre of the window's n - 1 range, plane spacing
    void *wx_d = nullptr, *wcorr_d = nullptr;  // [nb][nb] x' = n - 1 - x_c and 1/(n Phi(dw x'))
    void *wpairs_d = nullptr, *pv_d = nullptr;
    int wres_blocks = 0, nwpair = 0;
    std::vector<int> pair_slot0, pair_nslot, pair_widx;  // by pair index (wterm)
    // feathering
    void *feather_tw_d = nullptr, *feather_b1_d = nullptr;  // DFT twiddles and b1 of length n
    cudaGraphExec_t graph = nullptr;
    int launches = 0;
    bool capturing = false;
    bool any_grid = false;  // some pair uses a re-projection grid (set at prepare)
    // solver state
    SolverBufs solver{};
    // profiling
    bool profile = false;        // stage events wanted
    bool graph_profiled = false; // the instantiated graph carries stage events
    bool prof_pending = false;   // a profiled evaluation has not been accumulated yet
    Stage stages[MAX_STAGES]{};
    int nstage = 0;
    long long prof_evals = 0;
    std::string err;
};

namespace {

#define CK(call)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            return fail(p, IVIS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                           \
    } while (0)

ivis_status fail(ivis_plan_s *p, ivis_status s, const std::string &msg) {
    if (p) p->err = msg;
    else g_plan_error = msg;
    return s;
}

ivis_status alloc(ivis_plan_s *p, void **ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(p, IVIS_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                         cudaGetErrorString(e));
    }
    return IVIS_OK;
}

void dfree(void *&ptr) {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
}

// Order the plan's stream after everything already queued on the caller's stream.
void enter(ivis_plan_s *p) {
    cudaEventRecord(p->ev_in, p->user_stream);
    cudaStreamWaitEvent(p->stream, p->ev_in, 0);
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(long long v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

// ---------------------------------------------------------------- host-side NUFFT set-up
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Fourier transform of the ES kernel at integer frequency k of an nf grid:
// psi_hat(k) = int_{-W/2}^{W/2} psi(t) cos(2 pi k t / nf) dt.
void es_deapod(int nb, int nf, int W, double beta, std::vector<double> &dinv) {
    std::vector<double> zx, zw;
    gauss_legendre(200, zx, zw);
    dinv.resize(nb);
    for (int p = 0; p < nb; ++p) {
        int k = p - nb / 2;
        double acc = 0.0;
        for (size_t i = 0; i < zx.size(); ++i) {
            double z = zx[i];
            double phi = std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0));
            acc += zw[i] * phi * std::cos(M_PI * k * W * z / nf);
        }
        dinv[p] = 1.0 / (0.5 * W * acc);
    }
}

// w-stacking geometry of a window (Eq. 1): n - 1 over the window spans [x_min, 0] (corner to
// centre); x_c = x_min / 2, X = -x_min / 2, plane spacing dw = 1 / (4 X) (dw X <= 1/4, the
// oversampling-2 condition of the ES kernel). Per pixel: x' = n - 1 - x_c and
// corr = 1 / (n Phi(dw x')), Phi(xi) = int phi(t) cos(2 pi t xi) dt over t in [-W/2, W/2]
// (Gauss-Legendre, cached by the pixel's squared radius).
void w_tables(int nb, double cell, int W, double beta, double &xc, double &dw, std::vector<double> &wx,
              std::vector<double> &wcorr) {
    auto nm1 = [](double r2, double &n) { n = std::sqrt(1.0 - r2); return -r2 / (1.0 + n); };
    double ncorner;
    const double lc = 0.5 * nb * cell;
    const double xmin = nm1(2.0 * lc * lc, ncorner);
    xc = 0.5 * xmin;
    dw = 1.0 / (4.0 * (-0.5 * xmin));
    std::vector<double> zx, zw;
    gauss_legendre(200, zx, zw);
    const long long h = nb / 2;
    std::vector<double> cache((size_t)(2 * h * h + 1), -1.0);
    wx.resize((size_t)nb * nb);
    wcorr.resize((size_t)nb * nb);
    for (int q = 0; q < nb; ++q)
        for (int p = 0; p < nb; ++p) {
            const long long dq = q - h, dp = p - h, r2i = dq * dq + dp * dp;
            const double r2 = (double)r2i * cell * cell;
            double n;
            const double xp = nm1(r2, n) - xc;
            double &phi = cache[(size_t)r2i];
            if (phi < 0.0) {
                double acc = 0.0;
                for (size_t i = 0; i < zx.size(); ++i) {
                    const double z = zx[i];
                    acc += zw[i] * std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0)) * std::cos(M_PI * W * z * dw * xp);
                }
                phi = 0.5 * W * acc;
            }
            wx[(size_t)q * nb + p] = xp;
            wcorr[(size_t)q * nb + p] = 1.0 / (n * phi);
        }
}

// Per-tap polynomial of the ES kernel for the FP32 gridding kernels: for tap t and first-tap
// fraction f in [0, 1) the kernel argument is z = (f + W/2 - 1 - t) / (W/2); the value is
// interpolated at deg + 1 Chebyshev nodes in x = 2f - 1 and stored as monomial coefficients
// c[t][0..deg] (row stride ES_MAXDEG + 1) for Horner evaluation.
void es_fit(int W, double beta, int deg, std::vector<double> &c) {
    const int n = deg + 1;
    c.assign((size_t)W * (ES_MAXDEG + 1), 0.0);
    for (int t = 0; t < W; ++t) {
        std::vector<double> A((size_t)n * n), y(n);
        for (int k = 0; k < n; ++k) {
            const double x = std::cos(M_PI * (k + 0.5) / n);
            const double z = ((x + 1.0) * 0.5 + 0.5 * W - 1.0 - t) / (0.5 * W);
            const double a = 1.0 - z * z;
            y[k] = a >= 0.0 ? std::exp(beta * (std::sqrt(a) - 1.0)) : 0.0;
            double xp = 1.0;
            for (int i = 0; i < n; ++i) { A[(size_t)k * n + i] = xp; xp *= x; }
        }
        for (int col = 0; col < n; ++col) {  // Gaussian elimination, partial pivoting
            int piv = col;
            for (int r = col + 1; r < n; ++r)
                if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
            if (piv != col) {
                for (int i = 0; i < n; ++i) std::swap(A[(size_t)col * n + i], A[(size_t)piv * n + i]);
                std::swap(y[col], y[piv]);
            }
            for (int r = col + 1; r < n; ++r) {
                const double f = A[(size_t)r * n + col] / A[(size_t)col * n + col];
                for (int i = col; i < n; ++i) A[(size_t)r * n + i] -= f * A[(size_t)col * n + i];
                y[r] -= f * y[col];
            }
        }
        for (int i = n - 1; i >= 0; --i) {
            double acc = y[i];
            for (int j = i + 1; j < n; ++j) acc -= A[(size_t)i * n + j] * c[(size_t)t * (ES_MAXDEG + 1) + j];
            c[(size_t)t * (ES_MAXDEG + 1) + i] = acc / A[(size_t)i * n + i];
        }
    }
}

template <typename T>
ivis_status upload_real(ivis_plan_s *p, void **dst, const std::vector<double> &src) {
    std::vector<T> tmp(src.begin(), src.end());
    ivis_status s = alloc(p, dst, tmp.size() * sizeof(T));
    if (s) return s;
    CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return IVIS_OK;
}

// Twiddles of line_fft for lines of length L, in pass order: for each Stockham pass (Ns, R) the
// R x Ns block exp(-2 pi i k r / (Ns R)) at [16 (Ns - 1) / 15 + r Ns + k]; each value is
// exp(-2 pi i m / L) at m = k r L / (Ns R), computed in double and rounded once.
template <typename T>
std::vector<typename cplx_of<T>::type> fft_twiddles(int L) {
    typedef typename cplx_of<T>::type C;
    int logL = 0;
    while ((1 << logL) < L) ++logL;
    std::vector<C> tw;
    for (int logNs = 0; logNs < logL; logNs += 4) {
        const int R = 1 << std::min(4, logL - logNs), Ns = 1 << logNs;
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < Ns; ++k) {
                const long long m = (long long)k * r * (L / (Ns * R));
                const double a = 2.0 * M_PI * m / L;
                C w;
                w.x = (T)std::cos(a);
                w.y = (T)(-std::sin(a));
                tw.push_back(w);
            }
    }
    return tw;
}

template <typename T>
ivis_status upload_twiddles(ivis_plan_s *p) {
    typedef typename cplx_of<T>::type C;
    const std::vector<C> tw = fft_twiddles<T>(p->nf);
    ivis_status s = alloc(p, &p->tw_d, tw.size() * sizeof(C));
    if (s) return s;
    CK(cudaMemcpy(p->tw_d, tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice));
    return IVIS_OK;
}

// ------------------------------------------------------------------ kernel dispatch on W
// FP32 cost+gradient passes with kernel width <= 8 run k_grid_cg (one lane per kernel column);
// the FP64 path, wider kernels, the predict and spread-only modes run k_grid_pass.
inline bool use_grid_cg(const ivis_plan_s *p) { return !p->fp64 && p->W <= 8 && !p->cfg.wterm; }

template <typename T, int MODE, int TS>
cudaError_t launch_grid_pass_ts(ivis_plan_s *p, int first_chunk, int nchunk, double *jpart,
                                void *pred, int gfold) {
    typedef typename cplx_of<T>::type C;
    const Chunk *ch = p->chunks_d + first_chunk;
    const PairData<T> *pd = (const PairData<T> *)p->pdata_d;
    const C *F = (const C *)p->F;
    C *G = (C *)p->G;
    const int PW = TS + p->W - 1;
    size_t smem = (size_t)PW * PW * sizeof(C) * (MODE == MODE_COSTGRAD ? 2 : 1);
    T beta = (T)p->beta;
    const int ntx = p->nf / TS;
#define GP_CASE(WW)                                                                           \
    case WW: {                                                                                \
        auto kern = k_grid_pass<T, WW, MODE, TS>;                                             \
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
        kern<<<nchunk, 256, smem, p->stream>>>(ch, pd, F, G, p->lognf, ntx, p->f_half, gfold, \
                                               beta, p->kpoly_d, jpart, (C *)pred);           \
        break;                                                                                \
    }
    switch (p->W) {
        GP_CASE(2) GP_CASE(3) GP_CASE(4) GP_CASE(5) GP_CASE(6) GP_CASE(7) GP_CASE(8) GP_CASE(9)
        GP_CASE(10) GP_CASE(11) GP_CASE(12) GP_CASE(13) GP_CASE(14) GP_CASE(15) GP_CASE(16)
        default: return cudaErrorInvalidValue;
    }
#undef GP_CASE
    return cudaGetLastError();
}

// The item pass (k_grid_cg, or k_grid_tc with p->xkern == 2) over chunks [first, first + n)
// of the item work list (p->xchunks_d).
template <int TS>
cudaError_t launch_grid_cg_ts(ivis_plan_s *p, int first, int n, double *jpart, int gfold) {
#define CG_CASE(WW)                                                                                   \
    case WW: {                                                                                        \
        if (p->xkern == 2) {                                                                          \
            auto kern = k_grid_tc<WW, TS>;                                                            \
            const size_t sm = GridTC<WW, TS>::SMEM;                                                   \
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);         \
            kern<<<n, GridTC<WW, TS>::THREADS, sm, p->stream>>>(                                      \
                p->xchunks_d + first, p->items_d, (const PairData<float> *)p->pdata_d,                \
                (const float2 *)p->F, (float2 *)p->G, p->lognf, p->f_half, gfold, p->kpoly_d, jpart); \
            return cudaGetLastError();                                                                \
        }                                                                                             \
        auto kern = k_grid_cg<WW, TS>;                                                                \
        const size_t sm = GridCG<WW, TS>::SMEM;                                                       \
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);             \
        kern<<<n, GridCG<WW, TS>::THREADS, sm, p->stream>>>(                                          \
            p->xchunks_d + first, p->items_d, (const PairData<float> *)p->pdata_d, (const float2 *)p->F, \
            (float2 *)p->G, p->lognf, p->f_half, gfold, p->kpoly_d, jpart);                           \
        return cudaGetLastError();                                                                    \
    }
    switch (p->W) {
        CG_CASE(2) CG_CASE(3) CG_CASE(4) CG_CASE(5) CG_CASE(6) CG_CASE(7) CG_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef CG_CASE
}

// gfold: the adjoint grid is consumed by the packed adjoint column pass, which reads only the
// Hermitian part folded onto rows 0 .. nf/2.
template <typename T, int MODE>
cudaError_t launch_grid_pass(ivis_plan_s *p, int first_chunk, int nchunk, double *jpart,
                             void *pred, int gfold = 0) {
    if (nchunk <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (p->gtile == 64) return launch_grid_pass_ts<T, MODE, 64>(p, first_chunk, nchunk, jpart, pred, gfold);
    }
    return launch_grid_pass_ts<T, MODE, 32>(p, first_chunk, nchunk, jpart, pred, gfold);
}

// The cost+gradient grid pass for slots [slot0, slot0 + nslots): k_grid_cg on the item work
// list (FP32, W <= 8) or k_grid_pass on the tile work list. The pass writes one FP64 J partial
// per chunk at jpart + (the slot range's first chunk); returns the partials written in *nj.
bool packed_pass(const ivis_plan_s *p, int slot0, int nslots);

template <typename T>
cudaError_t launch_costgrad(ivis_plan_s *p, int slot0, int nslots, double *jpart, int *nj = nullptr) {
    const int gfold = packed_pass(p, slot0, nslots) ? 1 : 0;  // the adjoint of these slots is packed
    if (use_grid_cg(p)) {
        const int c0 = p->xchunk_first[slot0], n = p->xchunk_first[slot0 + nslots] - c0;
        if (nj) *nj = n;
        if (n <= 0) return cudaSuccess;
        return p->xtile == 64 ? launch_grid_cg_ts<64>(p, c0, n, jpart + c0, gfold)
                              : launch_grid_cg_ts<32>(p, c0, n, jpart + c0, gfold);
    }
    const int c0 = p->chunk_first[slot0], n = p->chunk_first[slot0 + nslots] - c0;
    if (nj) *nj = n;
    return launch_grid_pass<T, MODE_COSTGRAD>(p, c0, n, jpart + c0, nullptr, gfold);
}

// Number of FP64 J partials the cost+gradient pass of all slots writes.
int cost_partials(const ivis_plan_s *p) { return use_grid_cg(p) ? p->nxchunk : p->nchunk; }

void stage_begin(ivis_plan_s *p, const char *name, cudaStream_t st, int &si);
void stage_end(ivis_plan_s *p, cudaStream_t st, int &si);

// Row passes: 256 threads = lpb lines of nf/16 threads. Column passes: ncol x nf/16 threads.
// Forward passes for slots [slot0, slot0 + nslots) (all slots by default).
// Whole-plan passes over real windows (no w-planes) carry two slots per transform.
bool packed_pass(const ivis_plan_s *p, int slot0, int nslots) {
    return slot0 == 0 && nslots == p->nslot && !p->cfg.wterm && !p->cfg.serial_pairs;
}

// si: when given, the row and column passes of the packed path are recorded as two stages
// of the profiled graph (fwd_rows, fwd_cols).
template <typename T>
cudaError_t launch_forward(ivis_plan_s *p, const void *sky, int slot0 = 0, int nslots = -1, int *si = nullptr) {
    typedef typename cplx_of<T>::type C;
    const int nb = p->cfg.nb, nf = p->nf, tpl = nf / 16, lpb = 256 / tpl;
    if (nslots < 0) nslots = p->nslot;
    p->f_half = packed_pass(p, slot0, nslots) ? 1 : 0;  // read by the grid passes that follow
    if (packed_pass(p, slot0, nslots)) {
        const int npk = (nslots + 1) / 2, lc = std::max(0, p->logc_cols - 1);
        dim3 gr((nb + lpb - 1) / lpb, npk);
        size_t smem_row = (size_t)fft_smem_elems(nf, lpb) * sizeof(C);
        cudaFuncSetAttribute(k_fwd_rows_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
        if (si) stage_begin(p, "fwd_rows", p->stream, *si);
        k_fwd_rows_pk<T><<<gr, 256, smem_row, p->stream>>>(
            (const T *)sky, (const T *)p->wbeam_d, p->pinfo_d, nslots, (C *)p->rowbuf,
            p->cfg.n, nb, p->lognf, (const C *)p->tw_d, (const float2 *)p->grids_d);
        if (si) stage_end(p, p->stream, *si);
        dim3 gc(nf / (2 << lc), npk);
        size_t smem_col = (size_t)fft_smem_elems(nf, 2 << lc) * sizeof(C);
        cudaFuncSetAttribute(k_fwd_cols_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
        if (si) stage_begin(p, "fwd_cols", p->stream, *si);
        k_fwd_cols_pk<T><<<gc, tpl << (lc + 1), smem_col, p->stream>>>(
            (const C *)p->rowbuf, (C *)p->F, nslots, nb, p->lognf, lc, (const C *)p->tw_d);
        if (si) stage_end(p, p->stream, *si);
        return cudaGetLastError();
    }
    const PairInfo *pinfo = p->pinfo_d + slot0;
    C *rowbuf = (C *)p->rowbuf + (size_t)slot0 * nb * nf;
    C *F = (C *)p->F + (size_t)slot0 * nf * nf;
    dim3 gr((nb + lpb - 1) / lpb, nslots);
    size_t smem_row = (size_t)fft_smem_elems(nf, lpb) * sizeof(C);
    cudaFuncSetAttribute(k_fwd_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_fwd_rows<T><<<gr, 256, smem_row, p->stream>>>(
        (const T *)sky, (const T *)p->beams_d, pinfo, (const T *)p->dinv_d, rowbuf,
        p->cfg.n, nb, p->lognf, (const C *)p->tw_d, (const float2 *)p->grids_d, (const T *)p->wx_d,
        (const T *)p->wcorr_d);
    dim3 gc(nf >> p->logc_cols, nslots);
    size_t smem_col = (size_t)fft_smem_elems(nf, 1 << p->logc_cols) * sizeof(C);
    cudaFuncSetAttribute(k_fwd_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
    k_fwd_cols<T><<<gc, tpl << p->logc_cols, smem_col, p->stream>>>(
        (const C *)rowbuf, F, nb, p->lognf, p->logc_cols, (const C *)p->tw_d);
    return cudaGetLastError();
}

// Adjoint passes for slots [slot0, slot0 + nslots) (all slots by default). clear_st: when
// given, the packed path clears G on that stream (forked after the column pass; the caller
// joins p->ev_cjoin at the end of the evaluation), concurrently with the row pass and what
// follows it.
template <typename T>
cudaError_t launch_adjoint(ivis_plan_s *p, int slot0 = 0, int nslots = -1, int *si = nullptr,
                           cudaStream_t clear_st = nullptr) {
    typedef typename cplx_of<T>::type C;
    const int nb = p->cfg.nb, nf = p->nf, tpl = nf / 16, lpb = 256 / tpl;
    if (nslots < 0) nslots = p->nslot;
    if (packed_pass(p, slot0, nslots)) {
        const int npk = (nslots + 1) / 2, lc = std::max(0, p->logc_cols - 1);
        dim3 gc(nf / (2 << lc), npk);
        size_t smem_col = (size_t)fft_smem_elems(nf, 2 << lc) * sizeof(C);
        cudaFuncSetAttribute(k_adj_cols_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
        if (si) stage_begin(p, "adj_cols", p->stream, *si);
        k_adj_cols_pk<T><<<gc, tpl << (lc + 1), smem_col, p->stream>>>((C *)p->G, (C *)p->rowbuf, nslots, nb,
                                                                       p->lognf, lc, (const C *)p->tw_d);
        if (si) stage_end(p, p->stream, *si);
        // the read halves of G back to zero for the next gridding pass
        cudaStream_t cs = p->stream;
        if (clear_st) {
            cudaEventRecord(p->ev_cfork, p->stream);
            cudaStreamWaitEvent(clear_st, p->ev_cfork, 0);
            cs = clear_st;
        }
        if (si) stage_begin(p, "clear_G", cs, *si);
        k_clear_half<T><<<dim3(std::max(1, p->clear_blocks / nslots), nslots), 256, 0, cs>>>((C *)p->G, p->lognf);
        if (si) stage_end(p, cs, *si);
        if (clear_st) cudaEventRecord(p->ev_cjoin, clear_st);
        dim3 gr((nb + lpb - 1) / lpb, npk);
        size_t smem_row = (size_t)fft_smem_elems(nf, lpb) * sizeof(C);
        cudaFuncSetAttribute(k_adj_rows_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
        if (si) stage_begin(p, "adj_rows", p->stream, *si);
        k_adj_rows_pk<T><<<gr, 256, smem_row, p->stream>>>((const C *)p->rowbuf, (const T *)p->wbeam_d, p->pinfo_d,
                                                           nslots, (T *)p->contrib, p->cfg.n,
                                                           nb, p->lognf, (const C *)p->tw_d);
        if (si) stage_end(p, p->stream, *si);
        return cudaGetLastError();
    }
    C *G = (C *)p->G + (size_t)slot0 * nf * nf;
    C *rowbuf = (C *)p->rowbuf + (size_t)slot0 * nb * nf;
    T *contrib = (T *)p->contrib + (size_t)slot0 * nb * nb;
    dim3 gc(nf >> p->logc_cols, nslots);
    size_t smem_col = (size_t)fft_smem_elems(nf, 1 << p->logc_cols) * sizeof(C);
    cudaFuncSetAttribute(k_adj_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
    k_adj_cols<T><<<gc, tpl << p->logc_cols, smem_col, p->stream>>>(
        G, rowbuf, nb, p->lognf, p->logc_cols, (const C *)p->tw_d);
    dim3 gr((nb + lpb - 1) / lpb, nslots);
    size_t smem_row = (size_t)fft_smem_elems(nf, lpb) * sizeof(C);
    cudaFuncSetAttribute(k_adj_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_adj_rows<T><<<gr, 256, smem_row, p->stream>>>(
        rowbuf, (const T *)p->beams_d, p->pinfo_d + slot0, (const T *)p->dinv_d,
        contrib, p->cfg.n, nb, p->lognf, (const C *)p->tw_d, (const T *)p->wx_d, (const T *)p->wcorr_d);
    return cudaGetLastError();
}

// Toeplitz form of the data term for all slots: forward row DFTs of the windows (unit
// deapodisation), column DFT x spectrum x inverse column DFT, inverse row DFTs with the
// gradient, cost partials and the pairs' constants. Three launches.
template <typename T>
cudaError_t launch_toeplitz(ivis_plan_s *p) {
    typedef typename cplx_of<T>::type C;
    const int nb = p->cfg.nb, nf = p->nf, tpl = nf / 16, lpb = 256 / tpl;
    const int npk = (p->nslot + 1) / 2, lc = std::max(0, p->logc_cols - 1);
    C *rowbuf = (C *)p->rowbuf;
    dim3 gr((nb + lpb - 1) / lpb, npk);
    size_t smem_row = (size_t)fft_smem_elems(nf, lpb) * sizeof(C);
    cudaFuncSetAttribute(k_fwd_rows_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_fwd_rows_pk<T><<<gr, 256, smem_row, p->stream>>>(
        (const T *)p->x, (const T *)p->beams_d, p->pinfo_d, p->nslot, rowbuf,
        p->cfg.n, nb, p->lognf, (const C *)p->tw_d, (const float2 *)p->grids_d);
    dim3 gc(nf / (2 << lc), npk);
    size_t smem_col = (size_t)fft_smem_elems(nf, 2 << lc) * sizeof(C);
    cudaFuncSetAttribute(k_toep_cols_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
    k_toep_cols_pk<T><<<gc, tpl << (lc + 1), smem_col, p->stream>>>(
        rowbuf, (const T *const *)p->that_ptr_d, p->nslot, nb, p->lognf, lc, (const C *)p->tw_d);
    cudaFuncSetAttribute(k_toep_rows_pk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_toep_rows_pk<T><<<gr, 256, smem_row, p->stream>>>(
        rowbuf, (const T *)p->x, (const T *)p->beams_d, p->pinfo_d, p->nslot, (const T *const *)p->bwin_ptr_d,
        p->qconst_d, (T *)p->contrib, p->jpart, p->cfg.n, nb, p->lognf, (const C *)p->tw_d,
        (const float2 *)p->grids_d);
    return cudaGetLastError();
}

template <typename T>
size_t conv_smem(int R) {
    const size_t strip = std::max((size_t)(CONV_TO + 2 * R) * 33, (size_t)(CONV_SPLIT - 1) * CONV_NWO * CONV_OPT * 32);
    return (strip + 2 * R + 1) * sizeof(T);
}

template <typename T>
cudaError_t launch_fusion(ivis_plan_s *p, cudaStream_t st, const void *sky, void *tsd_out_e,
                          void *gradK_out, bool fused) {
    const int n = p->cfg.n, nchan = p->cfg.nchan, R = p->Rsd;
    if (p->sd_N) {
        // rows then columns, each a line DFT x taps' spectrum x inverse DFT
        typedef typename cplx_of<T>::type C;
        const int N = p->sd_N, tpl = N / 16, lpb = std::max(1, 256 / tpl), logc = p->sd_logc;
        const dim3 gr(((n + 1) / 2 + lpb - 1) / lpb, nchan), gc((n + (2 << logc) - 1) / (2 << logc), nchan);
        const size_t smr = (size_t)fft_smem_elems(N, lpb) * sizeof(C), smc = (size_t)fft_smem_elems(N, 1 << logc) * sizeof(C);
        cudaFuncSetAttribute(k_sdconv_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
        cudaFuncSetAttribute(k_sdconv_cols<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
        cudaFuncSetAttribute(k_sdconv_cols<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
        const T *sp = (const T *)p->sd_spec_d;
        const C *tw = (const C *)p->sd_tw_d;
        const int nt = lpb * tpl, ntc = tpl << logc;
        k_sdconv_rows<T><<<gr, nt, smr, st>>>((const T *)sky, (T *)p->tmp1, sp, n, p->sd_logN, tw);
        if (!fused) {
            k_sdconv_cols<T, 0><<<gc, ntc, smc, st>>>((const T *)p->tmp1, (T *)tsd_out_e, sp, n, p->sd_logN, logc, tw,
                                                      nullptr, nullptr, nullptr);
            return cudaGetLastError();
        }
        // the fused column pass leaves the column convolution of e; one row pass finishes B^T e
        k_sdconv_cols<T, 1><<<gc, ntc, smc, st>>>((const T *)p->tmp1, (T *)p->tmp2, sp, n, p->sd_logN, logc, tw,
                                                  (const T *)p->tsd_d, p->inv_sig2_d, p->kpart);
        k_sdconv_rows<T><<<gr, nt, smr, st>>>((const T *)p->tmp2, (T *)gradK_out, sp, n, p->sd_logN, tw);
        return cudaGetLastError();
    }
    const size_t sm = conv_smem<T>(R);
    cudaFuncSetAttribute(k_conv_axis<T, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_conv_axis<T, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_conv_axis<T, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 gr((n + 31) / 32, (n + CONV_TO - 1) / CONV_TO, nchan);
    const T *taps = (const T *)p->taps_d;
    k_conv_axis<T, 0, 0><<<gr, CONV_THREADS, sm, st>>>((const T *)sky, (T *)p->tmp1, taps, R, n, nullptr, nullptr, nullptr);
    if (!fused) {  // plain B (x) I into tsd_out_e
        k_conv_axis<T, 1, 0><<<gr, CONV_THREADS, sm, st>>>((const T *)p->tmp1, (T *)tsd_out_e, taps, R, n, nullptr,
                                                  nullptr, nullptr);
        return cudaGetLastError();
    }
    k_conv_axis<T, 1, 1><<<gr, CONV_THREADS, sm, st>>>((const T *)p->tmp1, (T *)p->tmp2, taps, R, n,
                                              (const T *)p->tsd_d, p->inv_sig2_d, p->kpart);
    k_conv_axis<T, 0, 0><<<gr, CONV_THREADS, sm, st>>>((const T *)p->tmp2, (T *)p->tmp1, taps, R, n, nullptr, nullptr, nullptr);
    k_conv_axis<T, 1, 0><<<gr, CONV_THREADS, sm, st>>>((const T *)p->tmp1, (T *)gradK_out, taps, R, n, nullptr,
                                              nullptr, nullptr);
    return cudaGetLastError();
}

// Stage intervals are recorded by external event nodes inside the profiled graph.
void stage_begin(ivis_plan_s *p, const char *name, cudaStream_t st, int &si) {
    if (!p->profile || si >= MAX_STAGES) return;
    p->stages[si].name = name;
    cudaEventRecordWithFlags(p->stages[si].b, st, cudaEventRecordExternal);
}
void stage_end(ivis_plan_s *p, cudaStream_t st, int &si) {
    if (!p->profile || si >= MAX_STAGES) return;
    cudaEventRecordWithFlags(p->stages[si].e, st, cudaEventRecordExternal);
    ++si;
    p->nstage = std::max(p->nstage, si);
}

// Enqueue one full evaluation at p->x into p->g and p->cost_d (and cost_h).
template <typename T>
cudaError_t enqueue_eval(ivis_plan_s *p, bool capture) {
    typedef typename cplx_of<T>::type C;
    cudaError_t e;
    const bool use_k = p->cfg.lambda_s != 0.0;
    const bool use_r = p->cfg.lambda_r != 0.0;
    int si = 0;
    int launches = 0;
    const bool fork = capture && use_k;
    bool cjoin = false;  // G cleared on side2: join before the end
    if (use_k) {
        cudaStream_t st = p->stream;
        if (fork) {
            cudaEventRecord(p->ev_fork, p->stream);
            cudaStreamWaitEvent(p->side, p->ev_fork, 0);
            st = p->side;
        }
        stage_begin(p, "fusion_K", st, si);
        if ((e = launch_fusion<T>(p, st, p->x, nullptr, p->gradK, true)) != cudaSuccess) return e;
        launches += p->sd_N ? 3 : 4;  // line-DFT passes, or the direct-tap passes
        stage_end(p, st, si);
        if (fork) cudaEventRecord(p->ev_join, p->side);
    }
    if (p->nslot > 0 && p->cfg.toeplitz) {
        stage_begin(p, "toeplitz_data_term", p->stream, si);
        if ((e = launch_toeplitz<T>(p)) != cudaSuccess) return e;
        launches += 3;
        stage_end(p, p->stream, si);
    } else if (p->nslot > 0 && p->cfg.wterm) {
        // w-stacking: interpolation from every plane, per-visibility residuals, spreading
        stage_begin(p, "fwd_fft", p->stream, si);
        if ((e = launch_forward<T>(p, p->x)) != cudaSuccess) return e;
        stage_end(p, p->stream, si);
        stage_begin(p, "w_interp", p->stream, si);
        if ((e = launch_grid_pass<T, MODE_PREDICT>(p, 0, p->nchunk, nullptr, p->pv_d)) != cudaSuccess) return e;
        stage_end(p, p->stream, si);
        stage_begin(p, "w_residual", p->stream, si);
        k_w_residual<T, false><<<dim3(p->wres_blocks, p->nwpair), 256, 0, p->stream>>>(
            (const WPair<T> *)p->wpairs_d, p->W, (const C *)p->pv_d, p->jpart, nullptr);
        stage_end(p, p->stream, si);
        stage_begin(p, "w_spread", p->stream, si);
        if ((e = launch_grid_pass<T, MODE_SPREAD>(p, 0, p->nchunk, nullptr, nullptr)) != cudaSuccess) return e;
        stage_end(p, p->stream, si);
        stage_begin(p, "adj_fft", p->stream, si);
        if ((e = launch_adjoint<T>(p)) != cudaSuccess) return e;
        stage_end(p, p->stream, si);
        launches += 7;
    } else if (p->nslot > 0) {
        // the adjoint grid is zero here: zeroed at prepare and by every adjoint column pass
        if (p->cfg.serial_pairs) {
            // one (pointing, channel) pair at a time: the unbatched reference path
            stage_begin(p, "serial_pairs", p->stream, si);
            for (int sl = 0; sl < p->nslot; ++sl) {
                int nc = 0;
                if ((e = launch_forward<T>(p, p->x, sl, 1)) != cudaSuccess) return e;
                if ((e = launch_costgrad<T>(p, sl, 1, p->jpart, &nc)) != cudaSuccess) return e;
                if ((e = launch_adjoint<T>(p, sl, 1)) != cudaSuccess) return e;
                launches += 4 + (nc > 0 ? 1 : 0);
            }
            stage_end(p, p->stream, si);
        } else {
            // one stage per kernel: fwd_rows, fwd_cols, degrid_spread, adj_cols, clear_G, adj_rows
            if ((e = launch_forward<T>(p, p->x, 0, -1, &si)) != cudaSuccess) return e;
            launches += 2;
            stage_begin(p, "degrid_spread", p->stream, si);
            if ((e = launch_costgrad<T>(p, 0, p->nslot, p->jpart)) != cudaSuccess) return e;
            launches += 1;
            stage_end(p, p->stream, si);
            if ((e = launch_adjoint<T>(p, 0, -1, &si, capture ? p->side2 : nullptr)) != cudaSuccess) return e;
            launches += 3;  // adjoint columns, clearing of G (beside the rows when captured), adjoint rows
            cjoin = capture;
        }
    }
    if (fork) cudaStreamWaitEvent(p->stream, p->ev_join, 0);
    const int n = p->cfg.n, nchan = p->cfg.nchan;
    stage_begin(p, "assemble_R", p->stream, si);
    {
        auto kas = assemble_te(n, nchan) == 16 ? k_assemble<T, 16> : k_assemble<T, 32>;
        kas<<<assemble_grid(n, nchan), 256, 0, p->stream>>>(
            (const T *)p->x, (const T *)p->contrib, p->pinfo_d, p->chan_start_d, p->chan_list_d,
            (const T *)p->gradK, (T *)p->g, n, p->cfg.nb, nchan, (T)p->cfg.lambda_r,
            (T)p->cfg.lambda_s, use_r ? 1 : 0, use_k ? 1 : 0, p->rpart);
    }
    launches += 1;
    if (p->any_grid && p->nslot > 0) {
        dim3 gs((p->cfg.nb * p->cfg.nb + 255) / 256, p->nslot);
        k_grid_scatter<T><<<gs, 256, 0, p->stream>>>((const T *)p->contrib, p->pinfo_d,
                                                     (const float2 *)p->grids_d, (T *)p->g, n, p->cfg.nb);
        launches += 1;
    }
    stage_end(p, p->stream, si);
    stage_begin(p, "finalize", p->stream, si);
    k_finalize<<<FIN_BLOCKS, 256, 0, p->stream>>>(p->jpart, (p->cfg.toeplitz || p->cfg.wterm) ? p->njpart : cost_partials(p), p->kpart,
                                         use_k ? p->nkpart : 0,
                                         p->rpart, use_r ? p->nrpart : 0, p->cfg.lambda_r,
                                         p->cfg.lambda_s, p->cost_d);
    launches += 1;
    stage_end(p, p->stream, si);
    // the clearing of G (side stream) overlaps the row pass, the joint sum and the reductions,
    // none of which touches G; the next evaluation's gridding starts after this join
    if (cjoin) cudaStreamWaitEvent(p->stream, p->ev_cjoin, 0);
    cudaMemcpyAsync(p->cost_h, p->cost_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    p->launches = launches;
    return cudaGetLastError();
}

cudaError_t enqueue_eval_any(ivis_plan_s *p, bool capture) {
    return p->fp64 ? enqueue_eval<double>(p, capture) : enqueue_eval<float>(p, capture);
}

ivis_status capture_graph(ivis_plan_s *p) {
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    cudaGraph_t gph;
    CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeRelaxed));
    p->capturing = true;
    p->nstage = 0;
    cudaError_t e = enqueue_eval_any(p, true);
    p->capturing = false;
    p->graph_profiled = p->profile;
    cudaError_t e2 = cudaStreamEndCapture(p->stream, &gph);
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e2));
    e = cudaGraphInstantiate(&p->graph, gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return IVIS_OK;
}

// Fold the stage events of the last profiled evaluation into the running totals.
ivis_status accumulate_profile(ivis_plan_s *p) {
    if (!p->prof_pending) return IVIS_OK;
    CK(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < p->nstage; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->stages[i].b, p->stages[i].e) == cudaSuccess) p->stages[i].ms += ms;
    }
    cudaGetLastError();
    p->prof_evals++;
    p->prof_pending = false;
    return IVIS_OK;
}

// Enqueue one evaluation at p->x (graph replay); with_sync waits and checks the cost.
ivis_status launch_eval(ivis_plan_s *p, bool with_sync) {
    ivis_status s;
    if ((s = accumulate_profile(p))) return s;
    if (p->graph_profiled != p->profile && (s = capture_graph(p))) return s;
    CK(cudaGraphLaunch(p->graph, p->stream));
    if (p->profile) p->prof_pending = true;
    if (!with_sync) return IVIS_OK;
    CK(cudaStreamSynchronize(p->stream));
    if (!std::isfinite(p->cost_h[0]))
        return fail(p, IVIS_ERR_NONFINITE, "non-finite cost");
    return IVIS_OK;
}

ivis_status run_eval(ivis_plan_s *p) { return launch_eval(p, true); }

template <typename T>
ivis_status set_vis_impl(ivis_plan_s *p, PairHost &ph, int m, const float *uvw, const float *vis,
                         const float *w) {
    typedef typename coord_of<T>::type CO;
    typedef typename cplx_of<T>::type C;
    const int nbins = p->nf * p->nf;  // one key per fine-grid cell (tile-major order)
    const int nsb = (nbins + 1023) / 1024;
    void *coord_tmp = nullptr, *key = nullptr, *cnt = nullptr, *cur = nullptr, *bsum = nullptr,
         *tst = nullptr, *err = nullptr;
    auto cleanup = [&]() { dfree(coord_tmp); dfree(key); dfree(cnt); dfree(cur); dfree(bsum); dfree(tst); dfree(err); };
    ivis_status s;
    if ((s = alloc(p, &coord_tmp, (size_t)m * sizeof(CO))) || (s = alloc(p, &key, (size_t)m * sizeof(int))) ||
        (s = alloc(p, &cnt, (size_t)nbins * sizeof(int))) || (s = alloc(p, &cur, (size_t)nbins * sizeof(int))) ||
        (s = alloc(p, &bsum, (size_t)nsb * sizeof(int))) || (s = alloc(p, &tst, (size_t)(nbins / 64 + 1) * sizeof(int))) ||
        (s = alloc(p, &err, sizeof(int)))) {
        cleanup();
        return s;
    }
    cudaMemsetAsync(err, 0, sizeof(int), p->stream);
    cudaMemsetAsync(cnt, 0, (size_t)nbins * sizeof(int), p->stream);
    const int nblk = (m + 255) / 256;
    const int ncb = nbins / 64;  // 8 x 8-cell blocks, 16 per sort bin
    const double scale = p->cfg.cell_rad * p->nf;
    k_vis_prepare<T><<<nblk, 256, 0, p->stream>>>(m, uvw, vis, w, scale, p->lognf, p->W, p->tile,
                                                   p->ntx, (CO *)coord_tmp, (int *)key, (int *)err);
    k_hist<<<nblk, 256, 0, p->stream>>>(m, (const int *)key, (int *)cnt);
    k_scan_block<<<nsb, 256, 0, p->stream>>>(nbins, (const int *)cnt, (int *)cur, (int *)bsum);
    k_scan_top<<<1, 1024, 0, p->stream>>>(nsb, (int *)bsum);
    k_scan_add<<<nsb, 256, 0, p->stream>>>(nbins, (int *)cur, (const int *)bsum);
    k_tile_starts<<<(ncb + 256) / 256, 256, 0, p->stream>>>(ncb, 64, m, (const int *)cur, (int *)tst);
    int herr = 0;
    ph.block_start.assign(ncb + 1, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ph.block_start.data(), tst, (size_t)(ncb + 1) * sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) { cleanup(); return fail(p, IVIS_ERR_CUDA, std::string("set_vis: ") + cudaGetErrorString(e)); }
    if (herr) { cleanup(); return fail(p, IVIS_ERR_NONFINITE, "set_vis: non-finite uvw/vis/weight or negative weight"); }
    ph.tile_count.assign(p->ntiles, 0);  // per sort bin (16 blocks)
    for (int t = 0; t < p->ntiles; ++t) ph.tile_count[t] = ph.block_start[16 * (t + 1)] - ph.block_start[16 * t];
    if ((s = alloc(p, &ph.coord, (size_t)m * sizeof(CO))) || (s = alloc(p, &ph.vis, (size_t)m * sizeof(C))) ||
        (s = alloc(p, &ph.w, (size_t)m * sizeof(T))) || (s = alloc(p, (void **)&ph.orig, (size_t)m * sizeof(int)))) {
        cleanup();
        return s;
    }
    k_vis_scatter<T><<<nblk, 256, 0, p->stream>>>(m, (const int *)key, (const CO *)coord_tmp, vis, w,
                                                   (int *)cur, (CO *)ph.coord, (C *)ph.vis, (T *)ph.w, ph.orig);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cleanup();
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("set_vis scatter: ") + cudaGetErrorString(e));
    ph.m = m;
    ph.set = true;
    return IVIS_OK;
}

// w-stacked visibilities of one pair (wterm = 1): plane range from the pair's w extent, W
// entries per visibility (plane k0 + t, weight phi(a - k)), sorted by (plane, tile, cell) with
// the same counting sort as set_vis_impl; per-visibility V, w, phase and weights kept in caller
// order for the residual kernel.
template <typename T>
ivis_status set_vis_w(ivis_plan_s *p, PairHost &ph, int m, const float *uvw, const float *vis,
                      const float *w) {
    typedef typename coord_of<T>::type CO;
    typedef typename cplx_of<T>::type C;
    const int W = p->W;
    ivis_status s;
    const int nbk = std::min(1024, (m + 255) / 256);
    void *mmd = nullptr, *coord_tmp = nullptr, *key = nullptr, *err = nullptr, *coord_e = nullptr,
         *key_e = nullptr, *cnt = nullptr, *cur = nullptr, *bsum = nullptr, *tst = nullptr;
    auto cleanup = [&]() {
        dfree(mmd); dfree(coord_tmp); dfree(key); dfree(err); dfree(coord_e); dfree(key_e);
        dfree(cnt); dfree(cur); dfree(bsum); dfree(tst);
    };
    if ((s = alloc(p, &mmd, 2 * nbk * sizeof(float)))) return s;
    k_w_minmax<<<nbk, 256, 0, p->stream>>>(m, uvw, (float *)mmd);
    std::vector<float> hmm(2 * nbk);
    {
        cudaError_t e0 = cudaGetLastError();
        if (e0 == cudaSuccess)
            e0 = cudaMemcpyAsync(hmm.data(), mmd, 2 * nbk * sizeof(float), cudaMemcpyDeviceToHost, p->stream);
        if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(p->stream);
        if (e0 != cudaSuccess) {
            cleanup();
            return fail(p, IVIS_ERR_CUDA, std::string("set_vis w range: ") + cudaGetErrorString(e0));
        }
    }
    double wmin = 1e300, wmax = -1e300;
    for (int b = 0; b < nbk; ++b) {
        wmin = std::min(wmin, (double)hmm[2 * b]);
        wmax = std::max(wmax, (double)hmm[2 * b + 1]);
    }
    if (!std::isfinite(wmin) || !std::isfinite(wmax) || wmin > wmax) {
        cleanup();
        return fail(p, IVIS_ERR_NONFINITE, "set_vis: non-finite w");
    }
    // half a plane of margin on each side keeps every visibility's W planes in [0, nplane)
    const double dw = p->w_dw;
    ph.w0 = wmin - (0.5 * W - 0.5) * dw;
    ph.nplane = (int)std::floor((wmax - wmin) / dw) + W + 1;
    const long long nf2 = (long long)p->nf * p->nf, E = (long long)m * W;
    if ((long long)ph.nplane * nf2 >= 0x7fffffffLL || E >= 0x7fffffffLL) {
        cleanup();
        return fail(p, IVIS_ERR_ARG, "set_vis: w range or visibility count too large for the w-planes");
    }
    const int nbins = (int)((long long)ph.nplane * nf2), nsb = (nbins + 1023) / 1024;
    const int ntt = ph.nplane * p->ntiles;
    if ((s = alloc(p, &coord_tmp, (size_t)m * sizeof(CO))) || (s = alloc(p, &key, (size_t)m * sizeof(int))) ||
        (s = alloc(p, &err, sizeof(int))) || (s = alloc(p, &coord_e, (size_t)E * sizeof(CO))) ||
        (s = alloc(p, &key_e, (size_t)E * sizeof(int))) || (s = alloc(p, &cnt, (size_t)nbins * sizeof(int))) ||
        (s = alloc(p, &cur, (size_t)nbins * sizeof(int))) || (s = alloc(p, &bsum, (size_t)nsb * sizeof(int))) ||
        (s = alloc(p, &tst, (size_t)(ntt + 1) * sizeof(int))) ||
        (s = alloc(p, &ph.v_wk, (size_t)E * sizeof(T))) || (s = alloc(p, &ph.v_phase, (size_t)m * sizeof(C))) ||
        (s = alloc(p, &ph.v_vis, (size_t)m * sizeof(C))) || (s = alloc(p, &ph.v_w, (size_t)m * sizeof(T)))) {
        cleanup();
        return s;
    }
    cudaMemsetAsync(err, 0, sizeof(int), p->stream);
    cudaMemsetAsync(cnt, 0, (size_t)nbins * sizeof(int), p->stream);
    const int nblk = (m + 255) / 256;
    const unsigned eblk = (unsigned)((E + 255) / 256);
    k_vis_prepare<T><<<nblk, 256, 0, p->stream>>>(m, uvw, vis, w, p->cfg.cell_rad * p->nf, p->lognf, W, p->tile,
                                                   p->ntx, (CO *)coord_tmp, (int *)key, (int *)err);
    k_w_entries<T><<<nblk, 256, 0, p->stream>>>(m, W, ph.nplane, uvw, vis, w, ph.w0, dw, p->w_xc, p->beta, nf2,
                                                 (const CO *)coord_tmp, (const int *)key, (CO *)coord_e,
                                                 (int *)key_e, (T *)ph.v_wk, (C *)ph.v_phase, (C *)ph.v_vis,
                                                 (T *)ph.v_w, (int *)err);
    k_hist<<<eblk, 256, 0, p->stream>>>((int)E, (const int *)key_e, (int *)cnt);
    k_scan_block<<<nsb, 256, 0, p->stream>>>(nbins, (const int *)cnt, (int *)cur, (int *)bsum);
    k_scan_top<<<1, 1024, 0, p->stream>>>(nsb, (int *)bsum);
    k_scan_add<<<nsb, 256, 0, p->stream>>>(nbins, (int *)cur, (const int *)bsum);
    k_tile_starts<<<(ntt + 256) / 256, 256, 0, p->stream>>>(ntt, p->tile * p->tile, (int)E, (const int *)cur,
                                                           (int *)tst);
    int herr = 0;
    std::vector<int> starts(ntt + 1, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(starts.data(), tst, (size_t)(ntt + 1) * sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) { cleanup(); return fail(p, IVIS_ERR_CUDA, std::string("set_vis: ") + cudaGetErrorString(e)); }
    if (herr) { cleanup(); return fail(p, IVIS_ERR_NONFINITE, "set_vis: non-finite uvw/vis/weight or negative weight"); }
    ph.plane_tile_count.assign(ntt, 0);
    for (int t = 0; t < ntt; ++t) ph.plane_tile_count[t] = starts[t + 1] - starts[t];
    ph.plane_start.assign(ph.nplane + 1, 0);
    for (int k = 0; k <= ph.nplane; ++k) ph.plane_start[k] = starts[(size_t)k * p->ntiles];
    if ((s = alloc(p, &ph.e_coord, (size_t)E * sizeof(CO))) || (s = alloc(p, &ph.e_val, (size_t)E * sizeof(C))) ||
        (s = alloc(p, &ph.e_w, (size_t)E * sizeof(T))) || (s = alloc(p, (void **)&ph.e_orig, (size_t)E * sizeof(int))) ||
        (s = alloc(p, (void **)&ph.e_pos, (size_t)E * sizeof(int)))) {
        cleanup();
        return s;
    }
    cudaMemsetAsync(ph.e_val, 0, (size_t)E * sizeof(C), p->stream);
    k_w_scatter<T><<<eblk, 256, 0, p->stream>>>(E, (const int *)key_e, (const CO *)coord_e, (const T *)ph.v_wk,
                                                 (int *)cur, (CO *)ph.e_coord, (T *)ph.e_w, ph.e_orig, ph.e_pos);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cleanup();
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("set_vis scatter: ") + cudaGetErrorString(e));
    ph.m = m;
    ph.set = true;
    return IVIS_OK;
}

// Toeplitz data of one pair (toeplitz = 1), from the caller's arrays: a plan with one
// pointing of window 2nb and unit beam over a 2nb x 2nb sky holds the pair twice, as channel 0
// with unit visibilities and as channel 1 with the data. Its gradient at I = 0 is
// -Re(F^H W 1) = -Re T on the offsets d in [-nb, nb)^2 (channel 0) and -Re(F^H W V) on the
// same window (channel 1, whose centre nb x nb is -b). The spectrum of the even cyclic
// embedding of Re T then comes from one nf x nf DFT; C from an FP64 sum over the data.
template <typename T>
ivis_status toeplitz_pair(ivis_plan_s *p, PairHost &ph, int m, const float *uvw, const float *vis,
                          const float *w) {
    typedef typename cplx_of<T>::type C;
    const int nb = p->cfg.nb, nf = p->nf, n2 = 2 * nb, tpl = nf / 16, lpb = 256 / tpl;
    ivis_status s;
    if (!p->toep_sub) {
        ivis_config c2 = p->cfg;
        c2.n = n2;
        c2.nchan = 2;
        c2.npoint = 1;
        c2.nb = n2;
        c2.lambda_r = c2.lambda_s = 0.0;
        c2.positivity = 0;
        c2.serial_pairs = 0;
        c2.autotune = 0;
        c2.toeplitz = 0;
        c2.grid_tile = 0;
        // T and b enter the cost multiplied by the data's energy C, which near a fit's optimum
        // exceeds Q by orders of magnitude: compute them with the widest kernel (FP64, about
        // 1e-15) or one cell wider than the plan's (FP32, at its rounding floor)
        c2.kernel_width = p->fp64 ? 16 : std::min(16, p->W + 1);
        ivis_plan_t sub = nullptr;
        if ((s = ivis_plan(&c2, p->stream, &sub))) return fail(p, s, "Toeplitz set-up plan: " + g_plan_error);
        p->toep_sub = sub;
        void *ones = nullptr;
        if ((s = alloc(p, &ones, (size_t)n2 * n2 * sizeof(float)))) return s;
        k_fill<float><<<(unsigned)(((size_t)n2 * n2 + 255) / 256), 256, 0, p->stream>>>((size_t)n2 * n2, 1.0f, (float *)ones);
        s = ivis_set_pointing(sub, 0, nb, nb, (const float *)ones);
        cudaStreamSynchronize(p->stream);
        dfree(ones);
        if (s) return fail(p, s, "Toeplitz set-up pointing: " + sub->err);
    }
    ivis_plan_s *sub = p->toep_sub;
    const size_t n22 = (size_t)n2 * n2;
    const int nblk_e = std::min(1024, (m + 255) / 256);
    void *uvis = nullptr, *zero = nullptr, *grad = nullptr, *buf = nullptr, *part = nullptr;
    auto cleanup = [&]() { dfree(uvis); dfree(zero); dfree(grad); dfree(buf); dfree(part); };
    if ((s = alloc(p, &uvis, (size_t)m * sizeof(float2))) || (s = alloc(p, &zero, 2 * n22 * sizeof(T))) ||
        (s = alloc(p, &grad, 2 * n22 * sizeof(T))) || (s = alloc(p, &buf, (size_t)nf * nf * sizeof(C))) ||
        (s = alloc(p, &part, (size_t)nblk_e * sizeof(double))) ||
        (s = alloc(p, &ph.that, (size_t)nf * nf * sizeof(T))) || (s = alloc(p, &ph.bwin, (size_t)nb * nb * sizeof(T)))) {
        cleanup();
        return s;
    }
    k_unit_vis<<<(m + 255) / 256, 256, 0, p->stream>>>(m, (float2 *)uvis);
    cudaMemsetAsync(zero, 0, 2 * n22 * sizeof(T), p->stream);
    k_vis_energy<<<nblk_e, 256, 0, p->stream>>>(m, vis, w, (double *)part);
    double cst = 0.0;
    if ((s = ivis_set_vis(sub, 0, 0, m, uvw, (const float *)uvis, w)) ||
        (s = ivis_set_vis(sub, 0, 1, m, uvw, vis, w)) ||
        (s = ivis_cost_grad(sub, zero, &cst, grad, nullptr))) {
        std::string msg = sub->err;
        cleanup();
        return fail(p, s, "Toeplitz set-up: " + msg);
    }
    const size_t smem_row = (size_t)fft_smem_elems(nf, lpb) * sizeof(C);
    cudaFuncSetAttribute(k_toep_embed_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_toep_embed_rows<T><<<(nf + lpb - 1) / lpb, 256, smem_row, p->stream>>>((const T *)grad, (T)-1, (C *)buf, p->lognf,
                                                                 (const C *)p->tw_d);
    const size_t smem_col = (size_t)fft_smem_elems(nf, 1 << p->logc_cols) * sizeof(C);
    cudaFuncSetAttribute(k_toep_embed_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
    k_toep_embed_cols<T><<<nf >> p->logc_cols, tpl << p->logc_cols, smem_col, p->stream>>>(
        (const C *)buf, (T *)ph.that, p->lognf, p->logc_cols, (T)(1.0 / ((double)nf * nf)), (const C *)p->tw_d);
    k_toep_crop<T><<<(nb * nb + 255) / 256, 256, 0, p->stream>>>((const T *)grad + n22, (T)-1, (T *)ph.bwin, nb);
    std::vector<double> hp(nblk_e);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, nblk_e * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cleanup();
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("Toeplitz set-up: ") + cudaGetErrorString(e));
    double sum = 0.0;
    for (double v : hp) sum += v;
    ph.qconst = 0.5 * sum;
    return IVIS_OK;
}

void free_pair(PairHost &ph) {
    dfree(ph.e_coord);
    dfree(ph.e_val);
    dfree(ph.e_w);
    {
        void *a = ph.e_orig, *b = ph.e_pos;
        dfree(a);
        dfree(b);
        ph.e_orig = ph.e_pos = nullptr;
    }
    dfree(ph.v_vis);
    dfree(ph.v_w);
    dfree(ph.v_phase);
    dfree(ph.v_wk);
    ph.nplane = 0;
    ph.plane_start.clear();
    ph.plane_tile_count.clear();
    ph.tile_count.clear();
    ph.block_start.clear();
    dfree(ph.that);
    dfree(ph.bwin);
    ph.qconst = 0.0;
    dfree(ph.coord);
    dfree(ph.vis);
    dfree(ph.w);
    void *o = ph.orig;
    dfree(o);
    ph.orig = nullptr;
    ph.set = false;
    ph.m = 0;
}

void release_prepared(ivis_plan_s *p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
    void *pi = p->pinfo_d, *ck = p->chunks_d, *cs = p->chan_start_d, *cl = p->chan_list_d;
    dfree(pi); dfree(p->pdata_d); dfree(ck); dfree(cs); dfree(cl);
    p->pinfo_d = nullptr; p->chunks_d = nullptr; p->chan_start_d = nullptr; p->chan_list_d = nullptr;
    void *xc = p->xchunks_d, *xi = p->items_d;
    dfree(xc); dfree(xi);
    p->xchunks_d = nullptr; p->items_d = nullptr;
    p->nxchunk = 0;
    dfree(p->taps_d);
    dfree(p->sd_spec_d);
    dfree(p->sd_tw_d);
    p->sd_N = 0;
    void *is = p->inv_sig2_d; dfree(is); p->inv_sig2_d = nullptr;
    dfree(p->rowbuf); dfree(p->F); dfree(p->G); dfree(p->contrib); dfree(p->wbeam_d);
    dfree(p->x); dfree(p->g); dfree(p->tmp1); dfree(p->tmp2); dfree(p->gradK);
    void *a = p->jpart, *b = p->kpart, *c = p->rpart, *d = p->cost_d;
    dfree(a); dfree(b); dfree(c); dfree(d);
    void *tp = p->that_ptr_d, *bp = p->bwin_ptr_d, *qc = p->qconst_d;
    dfree(tp); dfree(bp); dfree(qc);
    dfree(p->wpairs_d);
    dfree(p->pv_d);
    p->that_ptr_d = p->bwin_ptr_d = nullptr;
    p->qconst_d = nullptr;
    p->jpart = p->kpart = p->rpart = p->cost_d = nullptr;
    solver_free(p->solver);
    p->prepared = false;
}

// Work list of the grid pass: per slot, per non-empty tile (edge p->gtile), runs of at most
// cap visibilities. The sort bins are 32 x 32 cells in quad order (bin_of_tile), so a 64-cell
// tile is four consecutive bins.
constexpr int TUNE_CHUNKS[] = {256, 512, 1024, 2048};       // candidates with 32-cell tiles
constexpr int TUNE_CHUNKS64[] = {1024, 2048, 4096};         // candidates with 64-cell tiles
constexpr int TUNE_ITEMS[] = {16, 32, 64};                  // k_grid_cg: visibilities per item

void build_chunks(ivis_plan_s *p, int cap, std::vector<Chunk> &chunks, std::vector<int> &first) {
    chunks.clear();
    first.assign(p->nslot + 1, 0);
    const int per = p->gtile == 64 ? 4 : 1;  // sort bins per tile
    for (int sl = 0; sl < p->nslot; ++sl) {
        const int *tc = p->slot_tc[sl];
        first[sl] = (int)chunks.size();
        int acc = 0;
        for (int j = 0; j < p->ntiles; j += per) {
            int cnt = 0;
            for (int s = 0; s < per; ++s) cnt += tc[j + s];
            int t;
            if (per == 4) {
                t = j >> 2;  // quad index = row-major index of the 64-cell tile
            } else {
                int bx, by;
                tile_of_bin(j, p->ntx, bx, by);
                t = by * p->ntx + bx;
            }
            for (int b = 0; b < cnt; b += cap) chunks.push_back(Chunk{sl, t, acc + b, acc + std::min(cnt, b + cap)});
            acc += cnt;
        }
    }
    first[p->nslot] = (int)chunks.size();
}

// Work list of k_grid_cg: per slot, per tile of edge ts (row-major tiles), per non-empty 8 x 8
// block of the tile, items of at most len visibilities; chunks of at most GRID_ROUNDS rounds of
// ng items of one tile, each chunk's items sorted by decreasing length (the groups of a warp,
// which run in step, then get items of similar length). Blocks are 16 per 32-cell sort bin,
// bins in quad order (bin_of_tile).
constexpr int GRID_ROUNDS = 8;

void build_items(const ivis_plan_s *p, int ts, int len, std::vector<Chunk> &chunks, std::vector<Item> &items,
                 std::vector<int> &first) {
    chunks.clear();
    items.clear();
    first.assign(p->nslot + 1, 0);
    const int ng = (ts == 64 ? GridCG<7, 64>::NG : GridCG<7, 32>::NG) * GRID_ROUNDS;
    const int nbx = ts / 8;
    const int nt = p->nf / ts;
    for (int sl = 0; sl < p->nslot; ++sl) {
        const int *bs = p->slot_bs[sl];
        first[sl] = (int)chunks.size();
        for (int t = 0; t < nt * nt; ++t) {
            const int tyi = t / nt, txi = t - tyi * nt;
            const int i0 = (int)items.size();
            // the tile's 32-cell bins (one, or the four of a quad) and their 16 blocks each
            for (int sub = 0; sub < (ts == 64 ? 4 : 1); ++sub) {
                const int bx32 = ts == 64 ? 2 * txi + (sub & 1) : txi, by32 = ts == 64 ? 2 * tyi + (sub >> 1) : tyi;
                const int bin = bin_of_tile(bx32, by32, p->ntx);
                for (int bib = 0; bib < 16; ++bib) {
                    const int j = bin * 16 + bib;
                    const int b0 = bs[j], b1 = bs[j + 1];
                    const int bx = (ts == 64 ? 4 * (sub & 1) : 0) + (bib & 3);
                    const int by = (ts == 64 ? 4 * (sub >> 1) : 0) + (bib >> 2);
                    for (int v = b0; v < b1; v += len) items.push_back(Item{v, std::min(b1, v + len), by * nbx + bx, 0});
                }
            }
            const int i1 = (int)items.size();
            for (int c = i0; c < i1; c += ng) {
                const int ce = std::min(i1, c + ng);
                std::stable_sort(items.begin() + c, items.begin() + ce, [](const Item &x, const Item &y) {
                    return x.end - x.begin > y.end - y.begin;
                });
                chunks.push_back(Chunk{sl, t, c, ce});
            }
        }
    }
    first[p->nslot] = (int)chunks.size();
}

std::string tune_key(const ivis_plan_s *p) {
    long long m = 0;
    for (int sl = 0; sl < p->nslot; ++sl) m += p->slot_m[sl];
    int mb = 0;  // visibility-count class: power of two
    while ((1LL << mb) < m) ++mb;
    return "nf=" + std::to_string(p->nf) + " w=" + std::to_string(p->W) + " fp64=" + std::to_string((int)p->fp64) +
           " nslot=" + std::to_string(p->nslot) + " m2=" + std::to_string(mb) +
           (p->cfg.toeplitz ? " toeplitz" : "") + (p->cfg.wterm ? " wterm" : "");
}

// Autotuner: picks the grid-pass chunk size and the number of columns per CTA of the column
// FFT passes by timing candidates on this plan's data (CUDA events, after a warm-up launch).
// Decisions are cached per shape class in the file named by IVIS_AUTOTUNE_CACHE, if set.
// Build the k_grid_cg work list for (p->xtile, p->item_len) and copy it to the device arrays
// (sized at prepare for the longest candidate list).
ivis_status upload_items(ivis_plan_s *p) {
    std::vector<Chunk> ch;
    std::vector<Item> itv;
    build_items(p, p->xtile, p->item_len, ch, itv, p->xchunk_first);
    p->nxchunk = (int)ch.size();
    if (!ch.empty()) CK(cudaMemcpy(p->xchunks_d, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
    if (!itv.empty()) CK(cudaMemcpy(p->items_d, itv.data(), itv.size() * sizeof(Item), cudaMemcpyHostToDevice));
    return IVIS_OK;
}

template <typename T>
ivis_status autotune(ivis_plan_s *p) {
    ivis_status s_;
    const std::string key = tune_key(p);
    const char *path = std::getenv("IVIS_AUTOTUNE_CACHE");
    int best_cap = -1, best_logc = -1, best_ts = -1, best_kern = -1;
    if (path) {
        if (FILE *f = std::fopen(path, "r")) {
            char line[512];
            while (std::fgets(line, sizeof line, f)) {
                std::string l(line);
                const size_t bar = l.find('|');
                if (bar == std::string::npos || l.substr(0, bar) != key) continue;
                int cap = 0, lc = -1, ts = 32, kn = 1;
                const int got = std::sscanf(l.c_str() + bar + 1, "%d %d %d %d", &cap, &lc, &ts, &kn);
                if (got >= 2) {
                    best_cap = cap;
                    best_logc = lc;
                    best_ts = got >= 3 ? ts : 32;
                    best_kern = got >= 4 ? kn : 1;
                }
            }
            std::fclose(f);
        }
    }
    // tile edges the plan can use: 64 needs the FP32 path and at least 2 x 2 sort bins; a
    // tile fixed in the configuration is the only candidate
    auto tile_ok = [&](int ts) {
        if (p->cfg.grid_tile && ts != p->cfg.grid_tile) return false;
        return ts == 32 || (ts == 64 && !p->fp64 && p->ntx >= 2);
    };
    // chunk sizes (k_grid_pass) or visibilities per item (k_grid_cg) the tuner tries for a tile
    const bool cg = use_grid_cg(p);
    auto caps_of = [&](int ts) {
        if (cg) return std::vector<int>(std::begin(TUNE_ITEMS), std::end(TUNE_ITEMS));
        return ts == 64 ? std::vector<int>(std::begin(TUNE_CHUNKS64), std::end(TUNE_CHUNKS64))
                        : std::vector<int>(std::begin(TUNE_CHUNKS), std::end(TUNE_CHUNKS));
    };
    auto cap_ok = [&](int ts, int cap) {
        const std::vector<int> c = caps_of(ts);
        return std::find(c.begin(), c.end(), cap) != c.end();
    };
    // column-FFT widths the kernels can run: shared memory, threads per CTA, columns per grid
    const size_t csz = sizeof(typename cplx_of<T>::type);
    const int tpl = p->nf / 16;
    auto feasible_logc = [&](int lc) {
        return lc >= 0 && lc <= 4 && (size_t)fft_smem_elems(p->nf, 1 << lc) * csz <= 200 * 1024 &&
               (tpl << lc) <= (p->fp64 ? 512 : 1024) && (1 << lc) <= p->nf;
    };
    // a cached decision is used only if it is one the tuner itself could have made (the chunk
    // buffers are sized for the smallest candidate chunk)
    // item-pass kinds the plan can use: the configured one, else both
    auto kern_ok = [&](int k) { return cg && (k == 1 || k == 2) && (!p->cfg.grid_kernel || k == p->cfg.grid_kernel); };
    if (best_cap > 0 && (!tile_ok(best_ts) || !cap_ok(best_ts, best_cap) || !feasible_logc(best_logc) ||
                         (cg && !kern_ok(best_kern))))
        best_cap = best_logc = best_ts = best_kern = -1;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timed = [&](auto &&fn) -> float {
        fn();
        cudaEventRecord(e0, p->stream);
        for (int r = 0; r < 3; ++r) fn();
        cudaEventRecord(e1, p->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const bool cached = best_cap > 0 && best_logc >= 0;
    if (!cached) {
        // column-FFT width: the feasible values around the shared-memory default
        const int def = p->logc_cols;
        float bt = 1e30f;
        for (int lc = std::max(0, def - 1); lc <= std::min(4, def + 1); ++lc) {
            if (!feasible_logc(lc)) continue;
            p->logc_cols = lc;
            const float ms = timed([&] {
                if (p->cfg.toeplitz) {
                    launch_toeplitz<T>(p);
                } else {
                    launch_forward<T>(p, p->x);
                    launch_adjoint<T>(p);
                }
            });
            if (ms < bt) { bt = ms; best_logc = lc; }
        }
        // grid-pass tile edge (the sort bins the work list groups) and chunk size, or for
        // k_grid_cg the tile edge and the visibilities per item
        std::vector<Chunk> ch;
        std::vector<Item> itv;
        std::vector<int> first;
        float bg = 1e30f;
        for (int kn : {1, 2})
        for (int ts : {32, 64}) {
            if (!tile_ok(ts) || (cg ? !kern_ok(kn) : kn != 1)) continue;
            for (int cap : caps_of(ts)) {
                float ms;
                if (cg) {
                    p->xkern = kn;
                    p->xtile = ts;
                    build_items(p, ts, cap, ch, itv, first);
                    CK(cudaMemcpy(p->xchunks_d, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
                    CK(cudaMemcpy(p->items_d, itv.data(), itv.size() * sizeof(Item), cudaMemcpyHostToDevice));
                    p->xchunk_first = first;
                    ms = timed([&] { launch_costgrad<T>(p, 0, p->nslot, p->jpart); });
                } else {
                    p->gtile = ts;
                    build_chunks(p, cap, ch, first);
                    CK(cudaMemcpy(p->chunks_d, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
                    const int n = (int)ch.size();
                    ms = timed([&] {
                        if (p->cfg.wterm) {
                            launch_grid_pass<T, MODE_PREDICT>(p, 0, n, nullptr, p->pv_d);
                            launch_grid_pass<T, MODE_SPREAD>(p, 0, n, nullptr, nullptr);
                        } else {
                            launch_grid_pass<T, MODE_COSTGRAD>(p, 0, n, p->jpart, nullptr,
                                                               packed_pass(p, 0, p->nslot) ? 1 : 0);
                        }
                    });
                }
                if (ms < bg) { bg = ms; best_cap = cap; best_ts = ts; best_kern = kn; }
            }
        }
        CK(cudaGetLastError());
        if (path) {
            if (FILE *f = std::fopen(path, "a")) {
                std::fprintf(f, "%s|%d %d %d %d\n", key.c_str(), best_cap, best_logc, best_ts, best_kern);
                std::fclose(f);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->logc_cols = best_logc;
    std::string grid;
    if (cg) {
        p->xkern = best_kern;
        p->xtile = best_ts;
        p->item_len = best_cap;
        if ((s_ = upload_items(p))) return s_;
        grid = std::string(p->xkern == 2 ? "tensor-core" : "scalar") + " item pass, tile " +
               std::to_string(p->xtile) + ", items of " + std::to_string(p->item_len);
    } else {
        p->chunk_cap = best_cap;
        p->gtile = best_ts;
        std::vector<Chunk> ch;
        build_chunks(p, p->chunk_cap, ch, p->chunk_first);
        p->nchunk = (int)ch.size();
        CK(cudaMemcpy(p->chunks_d, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
        grid = "tile " + std::to_string(p->gtile) + ", chunk " + std::to_string(p->chunk_cap);
    }
    CK(cudaMemsetAsync(p->G, 0, (size_t)p->nslot * p->nf * p->nf * sizeof(typename cplx_of<T>::type), p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->tuned = key + " -> " + grid + ", fft columns per CTA " +
               std::to_string(1 << p->logc_cols) + (cached ? " (cached)" : " (timed)");
    return IVIS_OK;
}

template <typename T>
ivis_status prepare_impl(ivis_plan_s *p) {
    typedef typename cplx_of<T>::type C;
    const ivis_config &c = p->cfg;
    ivis_status s;
    for (int k = 0; k < c.npoint; ++k)
        if (!p->pset[k]) return fail(p, IVIS_ERR_STATE, "pointing " + std::to_string(k) + " not set");
    for (size_t i = 0; i < p->pairs.size(); ++i)
        if (!p->pairs[i].set)
            return fail(p, IVIS_ERR_STATE, "visibilities of pair (k=" + std::to_string(i % c.npoint) +
                                               ", chan=" + std::to_string(i / c.npoint) + ") not set");
    if (c.lambda_s != 0.0)
        for (int ch = 0; ch < c.nchan; ++ch)
            if (!p->sdset[ch]) return fail(p, IVIS_ERR_STATE, "single-dish map of channel " + std::to_string(ch) + " not set");
    // slots: pairs with data, in (chan, k) order; with the w-term, one slot per non-empty
    // w-plane of each such pair
    p->slot_pair.clear();
    p->slot_tc.clear();
    p->slot_bs.clear();
    p->slot_m.clear();
    std::vector<PairInfo> pinfo;
    std::vector<PairData<T>> pdata;
    std::vector<WPair<T>> wpairs;
    long long pv_total = 0;
    int max_m = 0;
    p->pair_slot0.assign(p->pairs.size(), 0);
    p->pair_nslot.assign(p->pairs.size(), 0);
    p->pair_widx.assign(p->pairs.size(), -1);
    typedef typename coord_of<T>::type CO;
    for (size_t i = 0; i < p->pairs.size(); ++i) {
        PairHost &ph = p->pairs[i];
        if (ph.m <= 0) continue;
        const int k = (int)(i % c.npoint), ch = (int)(i / c.npoint);
        p->pair_slot0[i] = (int)pinfo.size();
        if (!c.wterm) {
            pinfo.push_back(PairInfo{k, ch, p->cx[k], p->cy[k], p->pgrid[k], 0, 0.0});
            PairData<T> pd{};
            pd.coord = (const CO *)ph.coord;
            pd.vis = (const C *)ph.vis;
            pd.w = (const T *)ph.w;
            pd.orig = ph.orig;
            pd.m = ph.m;
            pd.pred_off = 0;
            pdata.push_back(pd);
            p->slot_pair.push_back((int)i);
            p->slot_tc.push_back(ph.tile_count.data());
            p->slot_bs.push_back(ph.block_start.data());
            p->slot_m.push_back(ph.m);
        } else {
            for (int pl = 0; pl < ph.nplane; ++pl) {
                const int b = ph.plane_start[pl], e = ph.plane_start[pl + 1];
                if (e <= b) continue;
                pinfo.push_back(PairInfo{k, ch, p->cx[k], p->cy[k], p->pgrid[k], 1, ph.w0 + pl * p->w_dw});
                PairData<T> pd{};
                pd.coord = (const CO *)ph.e_coord + b;
                pd.vis = (const C *)ph.e_val + b;
                pd.w = (const T *)ph.e_w + b;
                pd.orig = ph.e_orig + b;
                pd.m = e - b;
                pd.pred_off = pv_total;
                pdata.push_back(pd);
                p->slot_pair.push_back((int)i);
                p->slot_tc.push_back(ph.plane_tile_count.data() + (size_t)pl * p->ntiles);
                p->slot_bs.push_back(nullptr);
                p->slot_m.push_back(e - b);
            }
            WPair<T> wp{};
            wp.V = (const C *)ph.v_vis;
            wp.w = (const T *)ph.v_w;
            wp.phase = (const C *)ph.v_phase;
            wp.wk = (const T *)ph.v_wk;
            wp.epos = ph.e_pos;
            wp.ent_val = (C *)ph.e_val;
            wp.pv_off = pv_total;
            wp.m = ph.m;
            p->pair_widx[i] = (int)wpairs.size();
            wpairs.push_back(wp);
            pv_total += (long long)ph.m * p->W;
            max_m = std::max(max_m, ph.m);
        }
        p->pair_nslot[i] = (int)pinfo.size() - p->pair_slot0[i];
    }
    p->nslot = (int)pinfo.size();
    // per-slot kernels index the slot (or the two-window transform) on the grid's y dimension
    if (p->nslot > 65535)
        return fail(p, IVIS_ERR_ARG, "more than 65535 (pointing, channel) slots with data in one plan");
    std::vector<Chunk> chunks;
    std::vector<int> chan_start(c.nchan + 1, 0), chan_list;
    p->any_grid = false;
    for (int sl = 0; sl < p->nslot; ++sl) p->any_grid |= pinfo[sl].gridded != 0;
    build_chunks(p, p->chunk_cap, chunks, p->chunk_first);
    p->nchunk = (int)chunks.size();
    size_t max_chunks = 0;  // work lists of every autotuner candidate fit the device arrays
    {   // (32-cell tiles with the smallest chunk give the longest list)
        std::vector<Chunk> tmp;
        std::vector<int> tf;
        const int gt = p->gtile;
        p->gtile = 32;
        build_chunks(p, TUNE_CHUNKS[0], tmp, tf);
        p->gtile = gt;
        max_chunks = std::max(tmp.size(), chunks.size());
    }
    for (int ch = 0; ch < c.nchan; ++ch) {
        chan_start[ch] = (int)chan_list.size();
        for (int sl = 0; sl < p->nslot; ++sl)
            if (pinfo[sl].chan == ch) chan_list.push_back(sl);
    }
    chan_start[c.nchan] = (int)chan_list.size();
    auto up = [&](void **dst, const void *src, size_t bytes) -> ivis_status {
        ivis_status st = alloc(p, dst, bytes);
        if (st) return st;
        if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return IVIS_OK;
    };
    if ((s = up((void **)&p->pinfo_d, pinfo.data(), pinfo.size() * sizeof(PairInfo)))) return s;
    if ((s = up(&p->pdata_d, pdata.data(), pdata.size() * sizeof(PairData<T>)))) return s;
    if ((s = alloc(p, (void **)&p->chunks_d, max_chunks * sizeof(Chunk)))) return s;
    if (!chunks.empty()) CK(cudaMemcpy(p->chunks_d, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
    if (use_grid_cg(p)) {
        // item work list: device arrays sized for the longest candidate (32-cell tiles, the
        // shortest items), then the list of the current choice
        std::vector<Chunk> xc;
        std::vector<Item> xi;
        std::vector<int> xf;
        build_items(p, 32, TUNE_ITEMS[0], xc, xi, xf);
        const size_t mx_c = std::max<size_t>(1, xc.size()), mx_i = std::max<size_t>(1, xi.size());
        max_chunks = std::max(max_chunks, mx_c);
        if ((s = alloc(p, (void **)&p->xchunks_d, mx_c * sizeof(Chunk)))) return s;
        if ((s = alloc(p, (void **)&p->items_d, mx_i * sizeof(Item)))) return s;
        if ((s = upload_items(p))) return s;
    }
    if ((s = up((void **)&p->chan_start_d, chan_start.data(), chan_start.size() * sizeof(int)))) return s;
    if ((s = up((void **)&p->chan_list_d, chan_list.data(), chan_list.size() * sizeof(int)))) return s;
    const size_t nf2 = (size_t)p->nf * p->nf;
    const size_t npix = (size_t)c.nchan * c.n * c.n;
    if ((s = alloc(p, &p->rowbuf, (size_t)p->nslot * c.nb * p->nf * sizeof(C)))) return s;
    if ((s = alloc(p, &p->F, (size_t)p->nslot * nf2 * sizeof(C)))) return s;
    if ((s = alloc(p, &p->G, (size_t)p->nslot * nf2 * sizeof(C)))) return s;
    CK(cudaMemset(p->G, 0, (size_t)p->nslot * nf2 * sizeof(C)));
    if ((s = alloc(p, &p->contrib, (size_t)p->nslot * c.nb * c.nb * sizeof(T)))) return s;
    {   // beam x deapodisation per pointing, read by the packed row passes
        const size_t nw = (size_t)c.npoint * c.nb * c.nb;
        if ((s = alloc(p, &p->wbeam_d, nw * sizeof(T)))) return s;
        k_beam_deapod<T><<<(unsigned)((nw + 255) / 256), 256, 0, p->stream>>>(
            (const T *)p->beams_d, (const T *)p->dinv_d, c.nb, nw, (T *)p->wbeam_d);
        CK(cudaGetLastError());
    }
    if ((s = alloc(p, &p->x, npix * sizeof(T)))) return s;
    if ((s = alloc(p, &p->g, npix * sizeof(T)))) return s;
    size_t njp = std::max<size_t>(1, max_chunks);
    if (c.wterm && !wpairs.empty()) {
        p->wres_blocks = (max_m + 255) / 256;
        p->nwpair = (int)wpairs.size();
        p->njpart = p->nwpair * p->wres_blocks;
        njp = std::max<size_t>(njp, (size_t)p->njpart);
        if ((s = up(&p->wpairs_d, wpairs.data(), wpairs.size() * sizeof(WPair<T>)))) return s;
        if ((s = alloc(p, &p->pv_d, (size_t)pv_total * sizeof(C)))) return s;
    }
    if (c.toeplitz) {
        // per-slot spectrum and b pointers, constants; one partial per row-pass CTA
        const int lpb = 256 / (p->nf / 16);
        p->njpart = p->nslot * ((c.nb + lpb - 1) / lpb);
        njp = std::max<size_t>(njp, (size_t)p->njpart);
        std::vector<void *> tp(p->nslot), bp(p->nslot);
        std::vector<double> qc(p->nslot);
        for (int sl = 0; sl < p->nslot; ++sl) {
            const PairHost &ph = p->pairs[p->slot_pair[sl]];
            if (!ph.that || !ph.bwin) return fail(p, IVIS_ERR_STATE, "Toeplitz data of a pair missing");
            tp[sl] = ph.that;
            bp[sl] = ph.bwin;
            qc[sl] = ph.qconst;
        }
        if ((s = up((void **)&p->that_ptr_d, tp.data(), tp.size() * sizeof(void *)))) return s;
        if ((s = up((void **)&p->bwin_ptr_d, bp.data(), bp.size() * sizeof(void *)))) return s;
        if ((s = up((void **)&p->qconst_d, qc.data(), qc.size() * sizeof(double)))) return s;
        if (p->toep_sub) {  // its buffers are not needed until the next ivis_set_vis
            ivis_destroy(p->toep_sub);
            p->toep_sub = nullptr;
        }
    }
    if ((s = alloc(p, (void **)&p->jpart, njp * sizeof(double)))) return s;
    {
        const dim3 ag = assemble_grid(c.n, c.nchan);  // one R partial per k_assemble CTA
        p->nrpart = (int)(ag.x * ag.y);
    }
    if ((s = alloc(p, (void **)&p->rpart, (size_t)p->nrpart * sizeof(double)))) return s;
    if ((s = alloc(p, (void **)&p->cost_d, FIN_WORDS * sizeof(double)))) return s;
    CK(cudaMemset(p->cost_d, 0, FIN_WORDS * sizeof(double)));  // the reduction's ticket starts at 0
    // single dish: taps with a common half-width, per-channel 1/sigma^2
    bool need_sd = false;
    for (int ch = 0; ch < c.nchan; ++ch) need_sd |= (bool)p->sdset[ch];
    if (need_sd) {
        int R = 0;
        for (int ch = 0; ch < c.nchan; ++ch) {
            double sg = p->fwhm_sd[ch] / (2.0 * std::sqrt(2.0 * std::log(2.0)));
            R = std::max(R, (int)std::ceil(4.0 * sg));
        }
        p->Rsd = R;
        std::vector<double> taps((size_t)c.nchan * (2 * R + 1), 0.0), is2(c.nchan, 0.0);
        for (int ch = 0; ch < c.nchan; ++ch) {
            if (!p->sdset[ch]) continue;
            double sg = p->fwhm_sd[ch] / (2.0 * std::sqrt(2.0 * std::log(2.0)));
            int r = (int)std::ceil(4.0 * sg);
            double sum = 0.0;
            for (int t = -r; t <= r; ++t) sum += std::exp(-0.5 * (t / sg) * (t / sg));
            for (int t = -r; t <= r; ++t)
                taps[(size_t)ch * (2 * R + 1) + R + t] = std::exp(-0.5 * (t / sg) * (t / sg)) / sum;
            is2[ch] = 1.0 / (p->sig_sd[ch] * p->sig_sd[ch]);
        }
        if ((s = upload_real<T>(p, &p->taps_d, taps))) return s;
        if ((s = up((void **)&p->inv_sig2_d, is2.data(), is2.size() * sizeof(double)))) return s;
        if ((s = alloc(p, &p->tmp1, npix * sizeof(T)))) return s;
        if ((s = alloc(p, &p->tmp2, npix * sizeof(T)))) return s;
        if ((s = alloc(p, &p->gradK, npix * sizeof(T)))) return s;
        p->nkpart = ((c.n + 31) / 32) * ((c.n + CONV_TO - 1) / CONV_TO) * c.nchan;
        // line-DFT convolution when the padded period fits one CTA's line (N <= 8192)
        p->sd_N = 0;
        int N = 16;
        while (N < c.n + R) N *= 2;
        if (N <= 8192) {
            typedef typename cplx_of<T>::type C;
            const int tpl = N / 16;
            int logc = 0;
            auto fits = [&](int l) {
                return (size_t)fft_smem_elems(N, 1 << l) * sizeof(C) <= 100 * 1024 &&
                       (tpl << l) <= (p->fp64 ? 512 : 1024) && (2 << l) <= std::max(2, c.n);
            };
            while (logc < 4 && fits(logc + 1)) ++logc;
            if ((size_t)fft_smem_elems(N, 1 << logc) * sizeof(C) <= 200 * 1024 &&
                (size_t)fft_smem_elems(N, std::max(1, 256 / tpl)) * sizeof(C) <= 200 * 1024) {
                std::vector<double> spec((size_t)c.nchan * N, 0.0), twd(2 * (size_t)N);
                for (int ch = 0; ch < c.nchan; ++ch) {
                    const double *b = taps.data() + (size_t)ch * (2 * R + 1) + R;  // b[0] at offset R
                    for (int k = 0; k < N; ++k) {
                        double acc = b[0];
                        for (int t = 1; t <= R; ++t) acc += 2.0 * b[t] * std::cos(2.0 * M_PI * (double)((long long)k * t % N) / N);
                        spec[(size_t)ch * N + k] = acc / N;
                    }
                }
                const std::vector<C> tw = fft_twiddles<T>(N);
                if ((s = upload_real<T>(p, &p->sd_spec_d, spec))) return s;
                if ((s = alloc(p, &p->sd_tw_d, tw.size() * sizeof(C)))) return s;
                CK(cudaMemcpy(p->sd_tw_d, tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice));
                p->sd_N = N;
                p->sd_logN = ilog2(N);
                p->sd_logc = logc;
                p->nkpart = (c.n + (2 << logc) - 1) / (2 << logc) * c.nchan;
            }
        }
        if (!p->sd_N && conv_smem<T>(R) > 220 * 1024)
            return fail(p, IVIS_ERR_ARG, "single-dish beam too wide for the convolution strip");
        if ((s = alloc(p, (void **)&p->kpart, (size_t)p->nkpart * sizeof(double)))) return s;
    }
    if (!p->kpart && (s = alloc(p, (void **)&p->kpart, sizeof(double)))) return s;
    if ((s = solver_alloc<T>(p->solver, npix))) return fail(p, s, "solver buffers: out of device memory");
    p->prepared = true;
    if (c.autotune && p->nslot > 0 && (s = autotune<T>(p))) { p->prepared = false; return s; }
    if ((s = capture_graph(p))) { p->prepared = false; return s; }
    return IVIS_OK;
}

ivis_status ensure_prepared(ivis_plan_s *p) {
    if (p->prepared) return IVIS_OK;
    release_prepared(p);
    ivis_status s = p->fp64 ? prepare_impl<double>(p) : prepare_impl<float>(p);
    if (s) release_prepared(p);
    return s;
}

void invalidate(ivis_plan_s *p) {
    if (p->prepared) release_prepared(p);
}

// ------------------------------------------------------------------------------- solver
template <typename T>
ivis_status solve_impl(ivis_plan_s *p, void *sky_dev, int maxiter, int m_hist, double pgtol,
                       double ftol, double f_target, ivis_solve_report *rep) {
    auto t0 = std::chrono::steady_clock::now();
    SolverBufs &B = p->solver;
    ivis_status s = solver_ensure<T>(B, m_hist);
    if (s) return fail(p, s, "solver buffers: out of device memory");
    const size_t n = B.npix;
    const size_t bytes = n * sizeof(T);
    const int pos = p->cfg.positivity ? 1 : 0;
    const int stride = 3 * B.mcap + 4;
    const unsigned nb = (unsigned)B.nblk;
    T *x = (T *)p->x, *g = (T *)p->g, *xk = (T *)B.xk, *gk = (T *)B.gk, *d = (T *)B.d;
    T *S = (T *)B.S, *Y = (T *)B.Y;
    CK(cudaMemcpyAsync(x, sky_dev, bytes, cudaMemcpyDeviceToDevice, p->stream));
    k_sol_project<T><<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(x, n, pos);
    CK(cudaMemsetAsync(B.scal, 0, 16 * sizeof(double), p->stream));
    if ((s = run_eval(p))) return s;
    double f = p->cost_h[0];
    int evals = 1, iters = 0, status = 1;
    double pg = 0.0;
    CK(cudaMemcpyAsync(xk, x, bytes, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaMemcpyAsync(gk, g, bytes, cudaMemcpyDeviceToDevice, p->stream));
    std::vector<int> order;
    const double c1 = 1e-4;
    for (int it = 0; it <= maxiter; ++it) {
        SlotList ord{};
        ord.m = (int)order.size();
        for (int t = 0; t < ord.m; ++t) ord.slot[t] = order[t];
        k_sol_dots<T><<<nb, 256, 0, p->stream>>>(n, xk, gk, pos, S, Y, ord, stride, B.part);
        k_sol_small<<<1, 1024, 0, p->stream>>>(B.nblk, stride, B.part, ord, B.SY, B.YY, B.mcap, B.coef, B.scal);
        k_sol_dir<T><<<nb, 256, 0, p->stream>>>(n, xk, gk, pos, S, Y, ord, B.coef, B.scal, d, stride, B.part);
        k_sol_sum<<<1, 256, 0, p->stream>>>(B.nblk, stride, B.part, B.scal, 1);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(B.scal_h, B.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
        const double gd = B.scal_h[1];
        pg = B.scal_h[2];
        const double gg = B.scal_h[3];
        if (pg <= pgtol || f <= f_target) { status = 0; break; }
        if (it == maxiter) { status = 1; break; }
        if (!(gd < 0.0) || !std::isfinite(gd)) {
            if (!order.empty()) { order.clear(); --it; continue; }
            status = 2;
            break;
        }
        double alpha = order.empty() ? std::min(1.0, 1.0 / std::sqrt(gg)) : 1.0;
        bool accepted = false;
        double fnew = f;
        for (int trial = 0; trial < 40; ++trial) {
            k_sol_trial<T><<<nb, 256, 0, p->stream>>>(n, xk, gk, d, alpha, pos, x, stride, B.part);
            k_sol_sum<<<1, 256, 0, p->stream>>>(B.nblk, stride, B.part, B.scal, 4);
            CK(cudaGetLastError());
            // one host wait per trial: the evaluation and the trial's g.(x - xk) together
            ivis_status es = launch_eval(p, false);
            ++evals;
            if (es) return es;
            CK(cudaMemcpyAsync(B.scal_h + 4, B.scal + 4, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
            CK(cudaStreamSynchronize(p->stream));
            if (!std::isfinite(p->cost_h[0])) es = IVIS_ERR_NONFINITE;
            fnew = p->cost_h[0];
            const double dd = B.scal_h[4];
            if (es == IVIS_OK && fnew <= f + c1 * dd && dd <= 0.0) { accepted = true; break; }
            if (dd == 0.0) break;  // the projected step no longer moves
            // safeguarded quadratic backtracking on phi(a) = f(P(x + a d))
            double anew = 0.5 * alpha;
            if (es == IVIS_OK && std::isfinite(fnew)) {
                const double den = 2.0 * (fnew - f - dd);
                if (den > 0.0) anew = -dd * alpha / den;
            }
            alpha = std::min(0.5 * alpha, std::max(0.1 * alpha, anew));
        }
        if (!accepted) {
            status = 2;
            CK(cudaMemcpyAsync(x, xk, bytes, cudaMemcpyDeviceToDevice, p->stream));
            break;
        }
        ++iters;
        // new correction pair
        int slot;
        if ((int)order.size() < m_hist) {
            std::vector<char> used(B.mcap, 0);
            for (int o : order) used[o] = 1;
            slot = 0;
            while (used[slot]) ++slot;
        } else {
            slot = order.front();
            order.erase(order.begin());
        }
        SlotList ou{};
        ou.m = (int)order.size() + 1;
        for (size_t t = 0; t < order.size(); ++t) ou.slot[t] = order[t];
        ou.slot[ou.m - 1] = slot;
        k_sol_update<T><<<nb, 256, 0, p->stream>>>(n, x, g, xk, gk, S, Y, slot, ou, stride, B.part);
        k_sol_update_small<<<1, 1024, 0, p->stream>>>(B.nblk, stride, B.part, slot, ou, B.SY, B.YY,
                                                     B.mcap, 2.2e-16, B.scal);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(B.scal_h + 5, B.scal + 5, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
        if (B.scal_h[5] != 0.0) order.push_back(slot);
        const double rel = (f - fnew) / std::max(std::max(std::fabs(f), std::fabs(fnew)), 1.0);
        f = fnew;
        if (rel <= ftol) { status = 0; break; }
    }
    CK(cudaMemcpyAsync(sky_dev, xk, bytes, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (rep) {
        rep->iterations = iters;
        rep->evaluations = evals;
        rep->f = f;
        rep->pg_inf = pg;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        rep->status = status;
    }
    if (status == 2 && iters == 0) return fail(p, IVIS_ERR_LINESEARCH, "line search found no decrease");
    return IVIS_OK;
}

}  // namespace

namespace {
// Model visibilities of one pair at p->x into out (caller order).
template <typename T>
cudaError_t predict_impl(ivis_plan_s *p, int pair, void *out) {
    typedef typename cplx_of<T>::type C;
    const int s0 = p->pair_slot0[pair], ns = p->pair_nslot[pair];
    cudaError_t e = launch_forward<T>(p, p->x, s0, ns);
    const int c0 = p->chunk_first[s0], nc = p->chunk_first[s0 + ns] - c0;
    if (!p->cfg.wterm) {
        if (e == cudaSuccess) e = launch_grid_pass<T, MODE_PREDICT>(p, c0, nc, nullptr, out);
        return e;
    }
    if (e == cudaSuccess) e = launch_grid_pass<T, MODE_PREDICT>(p, c0, nc, nullptr, p->pv_d);
    if (e != cudaSuccess) return e;
    const int wi = p->pair_widx[pair], m = p->pairs[pair].m;
    k_w_residual<T, true><<<(m + 255) / 256, 256, 0, p->stream>>>((const WPair<T> *)p->wpairs_d + wi, p->W,
                                                                  (const C *)p->pv_d, nullptr, (C *)out);
    return cudaGetLastError();
}

template <typename T>
ivis_status dirty_impl(ivis_plan_s *p, void *dirty_dev, void *beamw_dev) {
    typedef typename cplx_of<T>::type C;
    const int n = p->cfg.n, nchan = p->cfg.nchan;
    const size_t npix = (size_t)nchan * n * n;
    if (p->cfg.wterm) return fail(p, IVIS_ERR_STATE, "the dirty image is not available on a wterm plan");
    CK(cudaMemsetAsync(p->x, 0, npix * sizeof(T), p->stream));
    if (p->nslot > 0) {
        // at I = 0 the model visibilities vanish: the residual is -V and the data-term
        // gradient is the adjoint of -w V
        CK(cudaMemsetAsync(p->F, 0, (size_t)p->nslot * p->nf * p->nf * sizeof(C), p->stream));
        CK(cudaMemsetAsync(p->G, 0, (size_t)p->nslot * p->nf * p->nf * sizeof(C), p->stream));
        cudaError_t e = launch_costgrad<T>(p, 0, p->nslot, p->jpart);
        if (e == cudaSuccess) e = launch_adjoint<T>(p);
        if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("dirty: ") + cudaGetErrorString(e));
    }
    {
        auto kas = assemble_te(n, nchan) == 16 ? k_assemble<T, 16> : k_assemble<T, 32>;
        kas<<<assemble_grid(n, nchan), 256, 0, p->stream>>>(
            (const T *)p->x, (const T *)p->contrib, p->pinfo_d, p->chan_start_d, p->chan_list_d, nullptr,
            (T *)p->g, n, p->cfg.nb, nchan, (T)0, (T)0, 0, 0, p->rpart);
    }
    if (p->any_grid && p->nslot > 0) {
        dim3 gs((p->cfg.nb * p->cfg.nb + 255) / 256, p->nslot);
        k_grid_scatter<T><<<gs, 256, 0, p->stream>>>((const T *)p->contrib, p->pinfo_d,
                                                     (const float2 *)p->grids_d, (T *)p->g, n, p->cfg.nb);
    }
    k_scale<T><<<(unsigned)((npix + 255) / 256), 256, 0, p->stream>>>(npix, (const T *)p->g, (T)-1, (T *)dirty_dev);
    if (beamw_dev) {
        const int np = p->cfg.npoint;
        std::vector<int> hv(p->cx);
        hv.insert(hv.end(), p->cy.begin(), p->cy.end());
        hv.insert(hv.end(), p->pgrid.begin(), p->pgrid.end());
        int *dv = nullptr;
        ivis_status s;
        if ((s = alloc(p, (void **)&dv, hv.size() * sizeof(int)))) return s;
        cudaMemcpyAsync(dv, hv.data(), hv.size() * sizeof(int), cudaMemcpyHostToDevice, p->stream);
        k_beam_weight<T><<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, p->stream>>>(
            (const T *)p->beams_d, dv, dv + np, dv + 2 * np, np, n, p->cfg.nb, (T *)beamw_dev);
        if (p->grids_d) {
            dim3 gb((p->cfg.nb * p->cfg.nb + 255) / 256, np);
            k_beam_weight_grid<T><<<gb, 256, 0, p->stream>>>((const T *)p->beams_d, (const float2 *)p->grids_d,
                                                             dv + 2 * np, n, p->cfg.nb, (T *)beamw_dev);
        }
        cudaError_t e = cudaStreamSynchronize(p->stream);
        void *a = dv;
        dfree(a);
        if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("beam weight: ") + cudaGetErrorString(e));
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(p->stream));
    return IVIS_OK;
}

}  // namespace

namespace {
// Short-spacing correction by feathering (appendix): both separable passes of the Gaussian
// transfer function on the n x n grid.
template <typename T>
ivis_status feather_impl(ivis_plan_s *p, const void *int_dev, const float *sd_dev, double theta_pix,
                         double sd_scale, void *out_dev) {
    typedef typename cplx_of<T>::type C;
    const int n = p->cfg.n, nchan = p->cfg.nchan, logn = ilog2(n);
    ivis_status s;
    if (!p->feather_tw_d) {
        const std::vector<C> tw = fft_twiddles<T>(n);
        if ((s = alloc(p, &p->feather_tw_d, tw.size() * sizeof(C)))) return s;
        const cudaError_t e0 = cudaMemcpy(p->feather_tw_d, tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice);
        if (e0 != cudaSuccess || (s = alloc(p, &p->feather_b1_d, n * sizeof(T)))) {
            dfree(p->feather_tw_d);  // set up both tables again on the next call
            return e0 != cudaSuccess ? fail(p, IVIS_ERR_CUDA, std::string("feather twiddles: ") + cudaGetErrorString(e0)) : s;
        }
    }
    // b1 at the DFT frequency of each index, k = j / n or (j - n) / n cycles per pixel
    const double sig = theta_pix / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    std::vector<T> b1(n);
    for (int j = 0; j < n; ++j) {
        const double k = (j < (n + 1) / 2 ? j : j - n) / (double)n;
        b1[j] = (T)std::exp(-2.0 * M_PI * M_PI * sig * sig * k * k);
    }
    CK(cudaMemcpyAsync(p->feather_b1_d, b1.data(), n * sizeof(T), cudaMemcpyHostToDevice, p->stream));
    const int tpl = n / 16, lpb = 256 / tpl;
    dim3 gr((n / 2 + lpb - 1) / lpb, nchan);
    const size_t smem_row = (size_t)fft_smem_elems(n, lpb) * sizeof(C);
    cudaFuncSetAttribute(k_feather_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_feather_rows<T><<<gr, 256, smem_row, p->stream>>>((const T *)int_dev, sd_dev, (T)sd_scale,
                                                        (const T *)p->feather_b1_d, (T *)out_dev, n, logn,
                                                        (const C *)p->feather_tw_d);
    int logc = 0;
    auto fits = [&](int l) {
        return (size_t)fft_smem_elems(n, 1 << l) * sizeof(C) <= 100 * 1024 && (tpl << l) <= (p->fp64 ? 512 : 1024) &&
               (2 << l) <= n;
    };
    while (logc < 4 && fits(logc + 1)) ++logc;
    dim3 gc(n / (2 << logc), nchan);
    const size_t smem_col = (size_t)fft_smem_elems(n, 1 << logc) * sizeof(C);
    cudaFuncSetAttribute(k_feather_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col);
    k_feather_cols<T><<<gc, tpl << logc, smem_col, p->stream>>>((const T *)int_dev, (const T *)p->feather_b1_d,
                                                                (T *)out_dev, n, logn, logc,
                                                                (const C *)p->feather_tw_d);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(p->stream));
    return IVIS_OK;
}
}  // namespace

// ------------------------------------------------ allocation-free single-dish prediction
// Some callers cannot allocate device memory at the point where they need B (x) I: for
// example code that runs while the device allocator must not be touched (inside a region
// that a memory pool or an outside framework owns), or an embedded host that forbids runtime
// allocation after start-up. For them, ivis_sd_predict_noalloc keeps its scratch (the row-pass
// intermediate image and the beam taps) in this file-scope device array instead of
// plan-owned memory. Every device that loads the library holds the array until the process
// exits.
// Half-width limit: the direct-tap convolution keeps a strip of (32 + 2R) x 33 inputs plus the
// 2R + 1 taps in shared memory, within 220 KiB for R <= 812 (68 R + 1057 <= 56320 floats).
constexpr int NOALLOC_MAX_R = 812;
constexpr int NOALLOC_TAP_WORDS = 1632;                  // >= 2 NOALLOC_MAX_R + 1, 128-byte multiple
constexpr size_t NOALLOC_MAX_PIXELS = (size_t)1 << 20;   // n * n <= 1,048,576 per call
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_TAP_WORDS + NOALLOC_MAX_PIXELS];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
float *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mu;

ivis_status noalloc_fail(ivis_status s, const std::string &msg) {
    g_plan_error = msg;  // read by ivis_last_error(NULL)
    return s;
}

// Device address of the scratch array on the current device (looked up once per device).
ivis_status noalloc_scratch(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(IVIS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return noalloc_fail(IVIS_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return noalloc_fail(IVIS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (float *)ptr;
    }
    *out = g_noalloc_ptr[dev];
    return IVIS_OK;
}
}  // namespace

// ======================================================================= C ABI
extern "C" {

ivis_status ivis_plan(const ivis_config *cfg, void *stream, ivis_plan_t *out) {
    if (!cfg || !out) return fail(nullptr, IVIS_ERR_ARG, "null config or output pointer");
    *out = nullptr;
    const ivis_config &c = *cfg;
    if (c.n < 1 || c.nchan < 1 || c.npoint < 1) return fail(nullptr, IVIS_ERR_ARG, "n, nchan, npoint must be >= 1");
    if (!is_pow2(c.nb) || c.nb < 16 || c.nb > 2048) return fail(nullptr, IVIS_ERR_ARG, "nb must be a power of two in [16, 2048]");
    if (!(c.cell_rad > 0.0) || !std::isfinite(c.cell_rad)) return fail(nullptr, IVIS_ERR_ARG, "cell_rad must be > 0");
    if (c.precision != IVIS_FP64 && c.precision != IVIS_FP32) return fail(nullptr, IVIS_ERR_ARG, "precision must be IVIS_FP64 or IVIS_FP32");
    if (c.kernel_width != 0 && (c.kernel_width < 2 || c.kernel_width > 16)) return fail(nullptr, IVIS_ERR_ARG, "kernel_width must be 0 or in [2, 16]");
    if (c.kernel_width == 0 && !(c.nufft_tol > 0.0 && c.nufft_tol < 1.0)) return fail(nullptr, IVIS_ERR_ARG, "nufft_tol must be in (0, 1)");
    if (!std::isfinite(c.lambda_r) || !std::isfinite(c.lambda_s) || c.lambda_r < 0 || c.lambda_s < 0)
        return fail(nullptr, IVIS_ERR_NONFINITE, "lambda_r and lambda_s must be finite and >= 0");
    if (c.toeplitz && c.nb > 1024) return fail(nullptr, IVIS_ERR_ARG, "toeplitz needs nb <= 1024");
    if (c.toeplitz && c.serial_pairs) return fail(nullptr, IVIS_ERR_ARG, "toeplitz and serial_pairs are exclusive");
    if (c.wterm && (c.toeplitz || c.serial_pairs))
        return fail(nullptr, IVIS_ERR_ARG, "wterm excludes toeplitz and serial_pairs");
    if (c.wterm && 2.0 * (0.5 * c.nb * c.cell_rad) * (0.5 * c.nb * c.cell_rad) >= 0.25)
        return fail(nullptr, IVIS_ERR_ARG, "wterm: the window reaches too far from its centre (l^2 + m^2 >= 1/4)");
    ivis_plan_s *p = new (std::nothrow) ivis_plan_s();
    if (!p) return fail(nullptr, IVIS_ERR_OOM, "host allocation failed");
    p->cfg = c;
    p->user_stream = (cudaStream_t)stream;
    p->fp64 = c.precision == IVIS_FP64;
    p->rsz = p->fp64 ? 8 : 4;
    p->nf = 2 * c.nb;
    p->lognf = ilog2(p->nf);
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            p->clear_blocks = 8 * sms;
        cudaGetLastError();  // no device here: keep the default
    }
    if (!p->fp64 && p->nf > 4096) { delete p; return fail(nullptr, IVIS_ERR_ARG, "IVIS_FP32 supports nb <= 2048"); }
    if (c.kernel_width) p->W = c.kernel_width;
    else p->W = std::min(16, std::max(2, (int)std::ceil(-std::log10(c.nufft_tol)) + 1));
    p->beta = 2.30 * p->W;
    p->tile = GTILE;  // nf >= 32 always (nb >= 16)
    p->ntx = p->nf / p->tile;
    p->ntiles = p->ntx * p->ntx;
    if (c.grid_tile != 0 && c.grid_tile != 32 && c.grid_tile != 64) {
        delete p;
        return fail(nullptr, IVIS_ERR_ARG, "grid_tile must be 0, 32 or 64");
    }
    if (c.grid_kernel < 0 || c.grid_kernel > 2) {
        delete p;
        return fail(nullptr, IVIS_ERR_ARG, "grid_kernel must be 0, 1 or 2");
    }
    if (c.grid_tile == 64 && (p->fp64 || p->ntx < 2)) {
        delete p;
        return fail(nullptr, IVIS_ERR_ARG, "grid_tile 64 needs IVIS_FP32 and nb >= 32");
    }
    p->gtile = c.grid_tile ? c.grid_tile : 32;
    p->chunk_cap = p->gtile == 64 ? 2048 : 1024;
    p->xtile = c.grid_tile ? c.grid_tile : 32;
    p->item_len = 32;
    p->xkern = c.grid_kernel ? c.grid_kernel : 1;
    {
        // columns per CTA in the column FFT passes: as many as fit 100 KB of shared memory
        // and 1024 threads; at least 4 (32-byte row segments) if 160 KB allows it
        size_t csz = p->fp64 ? 16 : 8;
        const int tpl = p->nf / 16;
        auto fits = [&](int l, size_t budget) {
            return (size_t)fft_smem_elems(p->nf, 1 << l) * csz <= budget &&
                   (tpl << l) <= (p->fp64 ? 512 : 1024) &&
                   (1 << l) <= p->nf;
        };
        int logc = 0;
        while (logc < 4 && fits(logc + 1, 100 * 1024)) ++logc;
        while (logc < 2 && fits(logc + 1, 160 * 1024)) ++logc;
        if (!fits(logc, 200 * 1024)) { delete p; return fail(nullptr, IVIS_ERR_ARG, "grid too large"); }
        p->logc_cols = logc;
    }
    p->cx.assign(c.npoint, 0);
    p->cy.assign(c.npoint, 0);
    p->pset.assign(c.npoint, 0);
    p->pgrid.assign(c.npoint, 0);
    p->pairs.resize((size_t)c.npoint * c.nchan);
    p->sdset.assign(c.nchan, 0);
    p->sig_sd.assign(c.nchan, 1.0);
    p->fwhm_sd.assign(c.nchan, 0.0);
    ivis_status s = IVIS_OK;
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(nullptr, IVIS_ERR_CUDA, "stream creation failed");
    }
    es_deapod(c.nb, p->nf, p->W, p->beta, p->dinv_h);
    if (p->fp64) {
        s = upload_real<double>(p, &p->dinv_d, p->dinv_h);
        if (!s) s = upload_twiddles<double>(p);
    } else {
        s = upload_real<float>(p, &p->dinv_d, p->dinv_h);
        if (!s) s = upload_twiddles<float>(p);
    }
    if (!s) {
        std::vector<double> kp;
        es_fit(p->W, p->beta, std::min(p->W + 1, ES_MAXDEG), kp);  // the degree of es_deg<W>
        std::vector<float> kpf(kp.begin(), kp.end());
        s = alloc(p, (void **)&p->kpoly_d, kpf.size() * sizeof(float));
        if (!s && cudaMemcpy(p->kpoly_d, kpf.data(), kpf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            s = IVIS_ERR_CUDA;
    }
    if (!s) s = alloc(p, &p->beams_d, (size_t)c.npoint * c.nb * c.nb * p->rsz);
    if (!s) {
        if (cudaMemset(p->beams_d, 0, (size_t)c.npoint * c.nb * c.nb * p->rsz) != cudaSuccess) s = IVIS_ERR_CUDA;
    }
    if (!s) s = alloc(p, &p->tsd_d, (size_t)c.nchan * c.n * c.n * p->rsz);
    if (!s && c.wterm) {
        std::vector<double> wx, wcorr;
        w_tables(c.nb, c.cell_rad, p->W, p->beta, p->w_xc, p->w_dw, wx, wcorr);
        s = p->fp64 ? upload_real<double>(p, &p->wx_d, wx) : upload_real<float>(p, &p->wx_d, wx);
        if (!s) s = p->fp64 ? upload_real<double>(p, &p->wcorr_d, wcorr) : upload_real<float>(p, &p->wcorr_d, wcorr);
    }
    if (!s && cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess) s = IVIS_ERR_CUDA;
    if (!s && cudaStreamCreateWithFlags(&p->side2, cudaStreamNonBlocking) != cudaSuccess) s = IVIS_ERR_CUDA;
    if (!s && cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess) s = IVIS_ERR_CUDA;
    for (int i = 0; i < MAX_STAGES && !s; ++i)
        if (cudaEventCreate(&p->stages[i].b) != cudaSuccess || cudaEventCreate(&p->stages[i].e) != cudaSuccess)
            s = IVIS_ERR_CUDA;
    if (!s && cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) s = IVIS_ERR_CUDA;
    if (!s && cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) s = IVIS_ERR_CUDA;
    if (!s && cudaEventCreateWithFlags(&p->ev_cfork, cudaEventDisableTiming) != cudaSuccess) s = IVIS_ERR_CUDA;
    if (!s && cudaEventCreateWithFlags(&p->ev_cjoin, cudaEventDisableTiming) != cudaSuccess) s = IVIS_ERR_CUDA;
    if (!s && cudaMallocHost((void **)&p->cost_h, 4 * sizeof(double)) != cudaSuccess) s = IVIS_ERR_OOM;
    if (s) {
        g_plan_error = p->err.empty() ? "plan set-up failed" : p->err;
        ivis_destroy(p);
        return s;
    }
    *out = p;
    return IVIS_OK;
}

ivis_status ivis_set_pointing(ivis_plan_t p, int k, int cx, int cy, const float *beam_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (k < 0 || k >= p->cfg.npoint || !beam_dev) return fail(p, IVIS_ERR_ARG, "bad pointing index or null beam");
    enter(p);
    size_t nn = (size_t)p->cfg.nb * p->cfg.nb;
    char *dst = (char *)p->beams_d + (size_t)k * nn * p->rsz;
    if (p->fp64) k_f32_to<double><<<(unsigned)((nn + 255) / 256), 256, 0, p->stream>>>(beam_dev, (double *)dst, nn);
    else CK(cudaMemcpyAsync(dst, beam_dev, nn * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(p->stream));
    p->cx[k] = cx;
    p->cy[k] = cy;
    p->pset[k] = 1;
    invalidate(p);
    return IVIS_OK;
}

ivis_status ivis_set_pointing_grid(ivis_plan_t p, int k, const float *grid_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (k < 0 || k >= p->cfg.npoint) return fail(p, IVIS_ERR_ARG, "bad pointing index");
    enter(p);
    invalidate(p);
    if (!grid_dev) {
        p->pgrid[k] = 0;
        return IVIS_OK;
    }
    const size_t per = (size_t)p->cfg.nb * p->cfg.nb * 2 * sizeof(float);
    if (!p->grids_d) {
        ivis_status s = alloc(p, &p->grids_d, per * p->cfg.npoint);
        if (s) return s;
    }
    CK(cudaMemcpyAsync((char *)p->grids_d + per * k, grid_dev, per, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->pgrid[k] = 1;
    return IVIS_OK;
}

ivis_status ivis_set_vis(ivis_plan_t p, int k, int chan, int64_t m, const float *uvw_dev,
                         const float *vis_dev, const float *weight_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    // m + 1023 must stay within int (block counts of the per-visibility kernels)
    if (k < 0 || k >= p->cfg.npoint || chan < 0 || chan >= p->cfg.nchan || m < 0 || m > (int64_t)0x7fffffff - 1024)
        return fail(p, IVIS_ERR_ARG, "bad pair index or visibility count");
    if (m > 0 && (!uvw_dev || !vis_dev || !weight_dev)) return fail(p, IVIS_ERR_ARG, "null visibility pointer");
    enter(p);
    PairHost &ph = p->pairs[(size_t)chan * p->cfg.npoint + k];
    invalidate(p);
    free_pair(ph);
    if (m == 0) {
        ph.set = true;
        return IVIS_OK;
    }
    ivis_status s;
    if (p->cfg.wterm)
        s = p->fp64 ? set_vis_w<double>(p, ph, (int)m, uvw_dev, vis_dev, weight_dev)
                    : set_vis_w<float>(p, ph, (int)m, uvw_dev, vis_dev, weight_dev);
    else
        s = p->fp64 ? set_vis_impl<double>(p, ph, (int)m, uvw_dev, vis_dev, weight_dev)
                    : set_vis_impl<float>(p, ph, (int)m, uvw_dev, vis_dev, weight_dev);
    if (!s && p->cfg.toeplitz)
        s = p->fp64 ? toeplitz_pair<double>(p, ph, (int)m, uvw_dev, vis_dev, weight_dev)
                    : toeplitz_pair<float>(p, ph, (int)m, uvw_dev, vis_dev, weight_dev);
    if (s) free_pair(ph);
    return s;
}

ivis_status ivis_set_sd(ivis_plan_t p, int chan, const float *tsd_dev, double sigma_sd, double fwhm_pix) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (chan < 0 || chan >= p->cfg.nchan || !tsd_dev) return fail(p, IVIS_ERR_ARG, "bad channel or null map");
    if (!(sigma_sd > 0.0) || !std::isfinite(sigma_sd) || !(fwhm_pix > 0.0) || !std::isfinite(fwhm_pix))
        return fail(p, IVIS_ERR_ARG, "sigma_sd and fwhm_pix must be finite and > 0");
    enter(p);
    size_t nn = (size_t)p->cfg.n * p->cfg.n;
    char *dst = (char *)p->tsd_d + (size_t)chan * nn * p->rsz;
    if (p->fp64) k_f32_to<double><<<(unsigned)((nn + 255) / 256), 256, 0, p->stream>>>(tsd_dev, (double *)dst, nn);
    else CK(cudaMemcpyAsync(dst, tsd_dev, nn * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(p->stream));
    p->sdset[chan] = 1;
    p->sig_sd[chan] = sigma_sd;
    p->fwhm_sd[chan] = fwhm_pix;
    invalidate(p);
    return IVIS_OK;
}

ivis_status ivis_prepare(ivis_plan_t p) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    enter(p);
    return ensure_prepared(p);
}

ivis_status ivis_cost_grad(ivis_plan_t p, const void *sky_dev, double *cost_out, void *grad_dev,
                           double *terms_out) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_dev || !cost_out || !grad_dev) return fail(p, IVIS_ERR_ARG, "null sky, cost or gradient pointer");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    size_t bytes = (size_t)p->cfg.nchan * p->cfg.n * p->cfg.n * p->rsz;
    CK(cudaMemcpyAsync(p->x, sky_dev, bytes, cudaMemcpyDeviceToDevice, p->stream));
    if ((s = run_eval(p))) return s;
    CK(cudaMemcpyAsync(grad_dev, p->g, bytes, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    *cost_out = p->cost_h[0];
    if (terms_out) {
        terms_out[0] = p->cost_h[1];
        terms_out[1] = p->cost_h[2];
        terms_out[2] = p->cost_h[3];
    }
    return IVIS_OK;
}

ivis_status ivis_cost_grad_host(ivis_plan_t p, const void *sky_host, double *cost_out, void *grad_host,
                                double *terms_out) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_host || !cost_out || !grad_host) return fail(p, IVIS_ERR_ARG, "null sky, cost or gradient pointer");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    size_t bytes = (size_t)p->cfg.nchan * p->cfg.n * p->cfg.n * p->rsz;
    CK(cudaMemcpyAsync(p->x, sky_host, bytes, cudaMemcpyHostToDevice, p->stream));
    if ((s = run_eval(p))) return s;
    CK(cudaMemcpyAsync(grad_host, p->g, bytes, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    *cost_out = p->cost_h[0];
    if (terms_out) {
        terms_out[0] = p->cost_h[1];
        terms_out[1] = p->cost_h[2];
        terms_out[2] = p->cost_h[3];
    }
    return IVIS_OK;
}

ivis_status ivis_predict(ivis_plan_t p, const void *sky_dev, int k, int chan, void *vis_out_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_dev || !vis_out_dev) return fail(p, IVIS_ERR_ARG, "null pointer");
    if (k < 0 || k >= p->cfg.npoint || chan < 0 || chan >= p->cfg.nchan) return fail(p, IVIS_ERR_ARG, "bad pair index");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    const int pair = chan * p->cfg.npoint + k;
    if (p->pairs[pair].m <= 0) return IVIS_OK;  // no visibilities
    size_t bytes = (size_t)p->cfg.nchan * p->cfg.n * p->cfg.n * p->rsz;
    CK(cudaMemcpyAsync(p->x, sky_dev, bytes, cudaMemcpyDeviceToDevice, p->stream));
    cudaError_t e = p->fp64 ? predict_impl<double>(p, pair, vis_out_dev) : predict_impl<float>(p, pair, vis_out_dev);
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("predict: ") + cudaGetErrorString(e));
    CK(cudaStreamSynchronize(p->stream));
    return IVIS_OK;
}

ivis_status ivis_sd_predict(ivis_plan_t p, const void *sky_dev, void *out_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_dev || !out_dev) return fail(p, IVIS_ERR_ARG, "null pointer");
    enter(p);
    for (int ch = 0; ch < p->cfg.nchan; ++ch)
        if (!p->sdset[ch]) return fail(p, IVIS_ERR_STATE, "dish beam of channel " + std::to_string(ch) + " not set");
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    cudaError_t e = p->fp64 ? launch_fusion<double>(p, p->stream, sky_dev, out_dev, nullptr, false)
                            : launch_fusion<float>(p, p->stream, sky_dev, out_dev, nullptr, false);
    if (e != cudaSuccess) return fail(p, IVIS_ERR_CUDA, std::string("sd_predict: ") + cudaGetErrorString(e));
    CK(cudaStreamSynchronize(p->stream));
    return IVIS_OK;
}

ivis_status ivis_get_nufft_params(ivis_plan_t p, int *w, double *beta, int *nf) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (w) *w = p->W;
    if (beta) *beta = p->beta;
    if (nf) *nf = p->nf;
    return IVIS_OK;
}

ivis_status ivis_profile(ivis_plan_t p, int enable) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    ivis_status s = accumulate_profile(p);
    if (s) return s;
    p->profile = enable != 0;
    for (int i = 0; i < MAX_STAGES; ++i) p->stages[i].ms = 0.0;
    p->prof_evals = 0;
    return IVIS_OK;
}

ivis_status ivis_stage_times(ivis_plan_t p, const char **names, double *ms, int cap, int *count) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    ivis_status s = accumulate_profile(p);
    if (s) return s;
    if (count) *count = p->nstage;
    for (int i = 0; i < p->nstage && i < cap; ++i) {
        if (names) names[i] = p->stages[i].name;
        if (ms) ms[i] = p->prof_evals ? p->stages[i].ms / p->prof_evals : 0.0;
    }
    return IVIS_OK;
}

ivis_status ivis_get_stream(ivis_plan_t p, void **stream) {
    if (!p || !stream) return fail(p, IVIS_ERR_ARG, "null pointer");
    *stream = (void *)p->stream;
    return IVIS_OK;
}

ivis_status ivis_cost_grad_async(ivis_plan_t p, const void *sky_dev, void *grad_dev, double *cost_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_dev || !grad_dev || !cost_dev) return fail(p, IVIS_ERR_ARG, "null sky, gradient or cost pointer");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    size_t bytes = (size_t)p->cfg.nchan * p->cfg.n * p->cfg.n * p->rsz;
    CK(cudaMemcpyAsync(p->x, sky_dev, bytes, cudaMemcpyDeviceToDevice, p->stream));
    if ((s = launch_eval(p, false))) return s;
    CK(cudaMemcpyAsync(cost_dev, p->cost_d, 4 * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaMemcpyAsync(grad_dev, p->g, bytes, cudaMemcpyDeviceToDevice, p->stream));
    return IVIS_OK;
}

ivis_status ivis_tuning(ivis_plan_t p, int *chunk_cap, int *fft_cols, const char **text) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    if (chunk_cap) *chunk_cap = p->chunk_cap;
    if (fft_cols) *fft_cols = 1 << p->logc_cols;
    if (text) *text = p->tuned.c_str();
    return IVIS_OK;
}

ivis_status ivis_launches_per_eval(ivis_plan_t p, int *count) {
    if (!p || !count) return fail(p, IVIS_ERR_ARG, "null pointer");
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    *count = p->launches;
    return IVIS_OK;
}

ivis_status ivis_solve(ivis_plan_t p, void *sky_dev, int maxiter, int m_hist, double pgtol, double ftol,
                       ivis_solve_report *rep) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_dev || maxiter < 0 || m_hist < 1 || m_hist > 32 || !(pgtol >= 0) || !(ftol >= 0))
        return fail(p, IVIS_ERR_ARG, "bad solve arguments");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    return p->fp64 ? solve_impl<double>(p, sky_dev, maxiter, m_hist, pgtol, ftol, -HUGE_VAL, rep)
                   : solve_impl<float>(p, sky_dev, maxiter, m_hist, pgtol, ftol, -HUGE_VAL, rep);
}

ivis_status ivis_solve_target(ivis_plan_t p, void *sky_dev, int maxiter, int m_hist, double pgtol,
                              double ftol, double f_target, ivis_solve_report *rep) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!sky_dev || maxiter < 0 || m_hist < 1 || m_hist > 32 || !(pgtol >= 0) || !(ftol >= 0) || std::isnan(f_target))
        return fail(p, IVIS_ERR_ARG, "bad solve arguments");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    return p->fp64 ? solve_impl<double>(p, sky_dev, maxiter, m_hist, pgtol, ftol, f_target, rep)
                   : solve_impl<float>(p, sky_dev, maxiter, m_hist, pgtol, ftol, f_target, rep);
}

ivis_status ivis_dirty_image(ivis_plan_t p, void *dirty_dev, void *beamw_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!dirty_dev) return fail(p, IVIS_ERR_ARG, "null dirty image pointer");
    enter(p);
    ivis_status s = ensure_prepared(p);
    if (s) return s;
    return p->fp64 ? dirty_impl<double>(p, dirty_dev, beamw_dev) : dirty_impl<float>(p, dirty_dev, beamw_dev);
}

ivis_status ivis_feather(ivis_plan_t p, const void *int_dev, const float *sd_dev, double theta_rad,
                         double sd_scale, void *out_dev) {
    if (!p) return fail(nullptr, IVIS_ERR_ARG, "null plan");
    if (!int_dev || !sd_dev || !out_dev) return fail(p, IVIS_ERR_ARG, "null pointer");
    if (out_dev == int_dev) return fail(p, IVIS_ERR_ARG, "out must not alias the interferometric map");
    const int n = p->cfg.n;
    if (!is_pow2(n) || n < 16 || n > 4096) return fail(p, IVIS_ERR_ARG, "feathering needs n a power of two in [16, 4096]");
    if (!(theta_rad > 0.0) || !std::isfinite(theta_rad) || !std::isfinite(sd_scale))
        return fail(p, IVIS_ERR_ARG, "theta must be finite and > 0, sd_scale finite");
    enter(p);
    const double theta_pix = theta_rad / p->cfg.cell_rad;
    return p->fp64 ? feather_impl<double>(p, int_dev, sd_dev, theta_pix, sd_scale, out_dev)
                   : feather_impl<float>(p, int_dev, sd_dev, theta_pix, sd_scale, out_dev);
}

ivis_status ivis_reproject_grid(int nb, double cell_rad, double ra_k, double dec_k, double ra0, double dec0,
                                double crpix_x, double crpix_y, int sky_proj, float *grid_host) {
    if (!grid_host) return fail(nullptr, IVIS_ERR_ARG, "null grid pointer");
    if (sky_proj != IVIS_PROJ_SIN && sky_proj != IVIS_PROJ_TAN && sky_proj != IVIS_PROJ_ARC)
        return fail(nullptr, IVIS_ERR_ARG, "unknown sky projection");
    if (nb < 1 || !(cell_rad > 0.0) || !std::isfinite(cell_rad)) return fail(nullptr, IVIS_ERR_ARG, "nb >= 1 and cell_rad > 0 required");
    for (double a : {ra_k, dec_k, ra0, dec0, crpix_x, crpix_y})
        if (!std::isfinite(a)) return fail(nullptr, IVIS_ERR_ARG, "non-finite angle or reference pixel");
    // orthonormal frames (east, north, centre) at a direction, in equatorial coordinates
    auto frame = [](double ra, double dec, double e[3], double nn[3], double c[3]) {
        const double sa = std::sin(ra), ca = std::cos(ra), sd = std::sin(dec), cd = std::cos(dec);
        e[0] = -sa; e[1] = ca; e[2] = 0.0;
        nn[0] = -sd * ca; nn[1] = -sd * sa; nn[2] = cd;
        c[0] = cd * ca; c[1] = cd * sa; c[2] = sd;
    };
    double ek[3], nk[3], ck[3], e0[3], n0[3], c0[3];
    frame(ra_k, dec_k, ek, nk, ck);
    frame(ra0, dec0, e0, n0, c0);
    // the rotation from pointing-frame to sky-frame direction cosines
    double R[3][3];
    const double *src[3] = {ek, nk, ck}, *dst[3] = {e0, n0, c0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = dst[i][0] * src[j][0] + dst[i][1] * src[j][1] + dst[i][2] * src[j][2];
    const float qnan = std::numeric_limits<float>::quiet_NaN();
    for (int q = 0; q < nb; ++q)
        for (int p = 0; p < nb; ++p) {
            const double l = (p - nb / 2) * cell_rad, m = (q - nb / 2) * cell_rad, r2 = l * l + m * m;
            float *g = grid_host + ((size_t)q * nb + p) * 2;
            if (r2 >= 1.0) { g[0] = g[1] = qnan; continue; }
            const double n = std::sqrt(1.0 - r2);
            const double l1 = R[0][0] * l + R[0][1] * m + R[0][2] * n;
            const double m1 = R[1][0] * l + R[1][1] * m + R[1][2] * n;
            const double n1 = R[2][0] * l + R[2][1] * m + R[2][2] * n;
            double f = 1.0;  // (x, y) = f (l', m')
            if (sky_proj == IVIS_PROJ_ARC) {
                const double st = std::sqrt(l1 * l1 + m1 * m1);  // sin(theta)
                if (n1 <= -1.0 + 1e-12) { g[0] = g[1] = qnan; continue; }
                f = st > 1e-12 ? std::atan2(st, n1) / st : 1.0;
            } else {
                if (n1 <= 0.0) { g[0] = g[1] = qnan; continue; }
                if (sky_proj == IVIS_PROJ_TAN) f = 1.0 / n1;
            }
            g[0] = (float)(crpix_x + f * l1 / cell_rad);
            g[1] = (float)(crpix_y + f * m1 / cell_rad);
        }
    return IVIS_OK;
}

double ivis_rayleigh_jeans(double freq_hz) {
    // 2 k nu^2 / c^2 in W m^-2 Hz^-1 sr^-1 per kelvin -> Jy per square arcsecond
    const double k_b = 1.380649e-23, c = 299792458.0, arcsec = M_PI / (180.0 * 3600.0);
    return 2.0 * k_b * freq_hz * freq_hz / (c * c) / 1e-26 * arcsec * arcsec;
}

ivis_status ivis_sd_predict_noalloc(const float *sky_dev, int n, int nchan, double fwhm_pix,
                                    float *out_dev, void *stream) {
    if (!sky_dev || !out_dev) return noalloc_fail(IVIS_ERR_ARG, "null sky or output pointer");
    if (n < 1 || nchan < 1) return noalloc_fail(IVIS_ERR_ARG, "n and nchan must be >= 1");
    if (!(fwhm_pix > 0.0) || !std::isfinite(fwhm_pix)) return noalloc_fail(IVIS_ERR_ARG, "fwhm_pix must be finite and > 0");
    if ((size_t)n * n > NOALLOC_MAX_PIXELS)
        return noalloc_fail(IVIS_ERR_ARG, "image too large for the allocation-free path: n*n must be <= " +
                                              std::to_string(NOALLOC_MAX_PIXELS));
    const double sg = fwhm_pix / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const double rr = std::ceil(4.0 * sg);
    if (rr > NOALLOC_MAX_R)
        return noalloc_fail(IVIS_ERR_ARG, "dish beam too wide for the allocation-free path: ceil(4 sigma) must be <= " +
                                              std::to_string(NOALLOC_MAX_R) + " (FWHM <= 478 pixels)");
    const int R = (int)rr;
    const size_t sm = conv_smem<float>(R);
    if (sm > 220 * 1024) return noalloc_fail(IVIS_ERR_ARG, "dish beam too wide for the convolution strip");
    // the taps are copied from this function's stack and the call waits for its stream: it
    // cannot be recorded into a graph
    cudaStream_t cs = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(cs, &cap);
    if (e != cudaSuccess) return noalloc_fail(IVIS_ERR_CUDA, std::string("sd_predict_noalloc: ") + cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
        return noalloc_fail(IVIS_ERR_STATE, "sd_predict_noalloc: the stream is capturing; the call is synchronous and "
                                            "copies its taps from host memory, so it cannot be captured");
    float *scratch = nullptr;
    ivis_status st = noalloc_scratch(&scratch);
    if (st) return st;
    float *taps_d = scratch;                       // [2R + 1]
    float *mid_d = scratch + NOALLOC_TAP_WORDS;    // [n][n] row-pass output of one channel
    float taps[NOALLOC_TAP_WORDS];
    double sum = 0.0;
    for (int t = -R; t <= R; ++t) sum += std::exp(-0.5 * (t / sg) * (t / sg));
    for (int t = -R; t <= R; ++t) taps[R + t] = (float)(std::exp(-0.5 * (t / sg) * (t / sg)) / sum);
    e = cudaMemcpyAsync(taps_d, taps, (size_t)(2 * R + 1) * sizeof(float), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_axis<float, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_axis<float, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 gr((n + 31) / 32, (n + CONV_TO - 1) / CONV_TO, 1);
    for (int c = 0; c < nchan && e == cudaSuccess; ++c) {
        const float *in = sky_dev + (size_t)c * n * n;
        float *out = out_dev + (size_t)c * n * n;
        k_conv_axis<float, 0, 0><<<gr, CONV_THREADS, sm, cs>>>(in, mid_d, taps_d, R, n, nullptr, nullptr, nullptr);
        k_conv_axis<float, 1, 0><<<gr, CONV_THREADS, sm, cs>>>(mid_d, out, taps_d, R, n, nullptr, nullptr, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return noalloc_fail(IVIS_ERR_CUDA, std::string("sd_predict_noalloc: ") + cudaGetErrorString(e));
    return IVIS_OK;
}

ivis_status ivis_destroy(ivis_plan_t p) {
    if (!p) return IVIS_OK;
    if (p->stream) cudaStreamSynchronize(p->stream);
    release_prepared(p);
    for (auto &ph : p->pairs) free_pair(ph);
    dfree(p->dinv_d);
    dfree(p->tw_d);
    {
        void *kp = p->kpoly_d;
        dfree(kp);
        p->kpoly_d = nullptr;
    }
    dfree(p->beams_d);
    dfree(p->tsd_d);
    dfree(p->wx_d);
    dfree(p->wcorr_d);
    dfree(p->feather_tw_d);
    dfree(p->feather_b1_d);
    if (p->toep_sub) ivis_destroy(p->toep_sub);
    p->toep_sub = nullptr;
    dfree(p->grids_d);
    for (auto &st : p->stages) {
        if (st.b) cudaEventDestroy(st.b);
        if (st.e) cudaEventDestroy(st.e);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->ev_cfork) cudaEventDestroy(p->ev_cfork);
    if (p->ev_cjoin) cudaEventDestroy(p->ev_cjoin);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->side2) cudaStreamDestroy(p->side2);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->cost_h) cudaFreeHost(p->cost_h);
    delete p;
    return IVIS_OK;
}

const char *ivis_last_error(ivis_plan_t p) {
    return p ? p->err.c_str() : g_plan_error.c_str();
}

}  // extern "C"
