/*
 * ivis.h -- C ABI of the B300 (sm_103a) engine for Classic3D's cost and gradient.
 *
 * The engine evaluates, for a sky cube I[nchan][N][N] (row-major, y then x),
 *
 *   Q_tot(I) = Q(I) + lambda_s K(I) + lambda_r R(I)                    (paper Eq. 14)
 *
 * with the joint data term Q = sum_k J_k over every (pointing k, channel) pair
 * (Eqs. 5-6), J_k = 1/2 sum_j w_j |V~_j - V_j|^2, the model visibilities
 * V~ of the primary-beam-weighted window I'_k (Eqs. 2-3, w-term and n-term
 * neglected as the paper does by default; the full Eq. 1 with wterm = 1 in
 * ivis_config), the Laplacian regulariser R (Eqs. 7-8) and
 * the single-dish fusion term K (Eqs. 11-13); and its analytic gradient.
 * The bounded quasi-Newton solve of Eq. 10 (I >= 0 when positivity is on) runs
 * on the device.
 *
 * Conventions used by every call:
 *  - Window of pointing k: I'_k[q][p] = I[cy - nb/2 + q][cx - nb/2 + p] (zero off
 *    the sky), or its bilinear re-projection (ivis_set_pointing_grid); direction
 *    cosines l_p = (p - nb/2) cell, m_q = (q - nb/2) cell;
 *    V~_j = sum_{q,p} A_k[q][p] I'_k[q][p] exp(-2 pi i (u_j l_p + v_j m_q)).
 *  - Real arrays whose type follows the plan's precision ("real" below) are
 *    double for IVIS_FP64 and float for IVIS_FP32. Costs are always double.
 *  - Pointers named *_dev are device pointers, *_host host pointers. Input
 *    buffers are borrowed for the duration of the call; set_* calls copy what
 *    they keep into plan-owned device memory. The caller keeps ownership of
 *    everything it passes in.
 *  - All device work runs on the plan's own stream (ivis_get_stream), which each
 *    call first orders after the work already queued on the caller's stream given
 *    to ivis_plan. Each call returns after its work is complete, except where
 *    stated.
 *  - No call aborts the process or throws across the ABI. On error the call
 *    returns a non-zero ivis_status, ivis_last_error() describes it, and the
 *    plan remains valid for ivis_destroy (and, unless the status is
 *    IVIS_ERR_CUDA, for further calls).
 */
#ifndef IVIS_H
#define IVIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ivis_plan_s *ivis_plan_t;

typedef enum {
    IVIS_OK = 0,
    IVIS_ERR_ARG = 1,        /* invalid argument (sizes, indices, null pointers)           */
    IVIS_ERR_STATE = 2,      /* call out of order (e.g. cost before every pair is set)     */
    IVIS_ERR_OOM = 3,        /* device allocation failed                                   */
    IVIS_ERR_CUDA = 4,       /* a CUDA runtime call failed                                 */
    IVIS_ERR_TIMEOUT = 5,    /* a bounded device wait ran out                              */
    IVIS_ERR_NONFINITE = 6,  /* NaN / Inf in inputs or in a computed cost                  */
    IVIS_ERR_LINESEARCH = 7  /* the solver's line search found no decrease                 */
} ivis_status;

enum { IVIS_FP64 = 0, IVIS_FP32 = 1 };

typedef struct {
    int n;              /* sky is n x n pixels per channel                                 */
    int nchan;          /* spectral channels (independent images, Sect. 2)                 */
    int npoint;         /* mosaic pointings                                                */
    int nb;             /* pointing window nb x nb, power of two, 16 <= nb <= 2048         */
    double cell_rad;    /* pixel size (radians); the same grid for sky and windows         */
    int precision;      /* IVIS_FP64: all arithmetic double. IVIS_FP32: gridding, FFTs and
                           residuals in float; the cost terms are summed in float within a
                           thread (at most 64 visibilities or a few pixels) and a warp, then
                           in double across warps and CTAs; the solver's inner products and
                           line-search slopes are accumulated in double from the first term */
    double nufft_tol;   /* target relative accuracy of the NUFFT when kernel_width == 0    */
    int kernel_width;   /* ES kernel width w in grid cells (2..16); 0 = chosen from tol     */
    double lambda_r;    /* weight of R (Eq. 14)                                            */
    double lambda_s;    /* weight of K (Eq. 14)                                            */
    int positivity;     /* 1: bound I >= 0 in ivis_solve (Sect. 3.4)                       */
    int serial_pairs;   /* 1: process the (pointing, channel) pairs one at a time (the
                           unbatched reference path); 0: all pairs in each kernel launch     */
    int autotune;       /* 1: ivis_prepare times candidate grid-pass chunk sizes and column-
                           FFT widths on this plan's data and keeps the fastest (cached per
                           shape class in the file named by IVIS_AUTOTUNE_CACHE, if set)     */
    int toeplitz;       /* 1: evaluate the data term of Eq. 6 through the Toeplitz form of its
                           normal operator (exact in exact arithmetic; the expansion of Eq. 6
                           with Eqs. 3-5): per pair, Q = 1/2 z'Re(H)z - z'b + C with
                           z = A .* P x, H = F^H W F, b = Re(F^H W V), C = 1/2 sum w|V|^2.
                           H acts as a cyclic convolution of period 2 nb, so an evaluation does
                           two pruned FFT passes per pair and no pass over the visibilities.
                           ivis_set_vis then also computes, per pair, the real 2nb x 2nb
                           spectrum of Re H and the window b (adjoint NUFFTs on a 2nb window;
                           device memory 4 nb^2 + nb^2 reals per pair). Needs nb <= 1024;
                           excludes serial_pairs. ivis_predict and ivis_dirty_image keep the
                           NUFFT. The FP32 cost carries an absolute error of about 1e-6 C (the
                           NUFFT path's is about 1e-6 sqrt(C Q)), so close to a fit's optimum
                           its relative error is larger than the NUFFT path's.               */
    int wterm;          /* 1: the full visibility equation (Eq. 1): the w-term
                           exp(-2 pi i w (n - 1)) and the 1/n factor, n = sqrt(1 - l^2 - m^2),
                           l, m the window pixel offsets times cell_rad. Computed by w-stacking:
                           the factor is interpolated between w-planes with the ES kernel of
                           the uv gridding (same width and accuracy); per pair the planes span
                           its w range at a spacing 1 / (2 |x_min|), x_min = n - 1 at the
                           window corner. Each visibility is stored W times (once per plane of
                           its kernel support). Excludes toeplitz and serial_pairs; needs the
                           window within l^2 + m^2 < 1/4; ivis_dirty_image is not available. */
    int grid_tile;      /* edge (fine-grid cells) of the tiles of the gridding work list
                           (Eqs. 3-6: each tile's patch of the oversampled grids is staged in
                           shared memory): 0 = default (64 in FP32 with kernel_width <= 8,
                           else 32; with autotune = 1 the autotuner times both and keeps the
                           faster), 32, or 64 (FP32 only; needs nb >= 32). Any other value:
                           IVIS_ERR_ARG. The result does not depend on it beyond rounding.   */
    int grid_kernel;    /* the fused interpolation / residual / spreading pass of the FP32
                           cost and gradient (kernel_width <= 8, no wterm): 0 = default (the
                           scalar pass; with autotune = 1 the autotuner times both and keeps
                           the faster), 1 = scalar pass (one lane per kernel column,
                           per-group adjoint buffers in shared memory), 2 = tensor-core pass
                           (per 8 x 8 block of first taps, interpolation F^T Ky and spreading
                           Ky diag(w r) Kx^T as TF32 mma with split operands, FP32-accurate).
                           Ignored where the pass does not apply. Any other value:
                           IVIS_ERR_ARG. The result does not depend on it beyond rounding.   */
} ivis_config;

typedef struct {
    int iterations;     /* accepted quasi-Newton steps                                     */
    int evaluations;    /* cost+gradient evaluations                                       */
    double f;           /* final Q_tot                                                     */
    double pg_inf;      /* final projected-gradient infinity norm                          */
    double seconds;     /* wall time of the solve                                          */
    int status;         /* 0 converged (pgtol/ftol), 1 maxiter reached, 2 line search stop */
} ivis_solve_report;

/* Create a plan. stream: a cudaStream_t (NULL = the legacy default stream). Every field of
 * cfg is checked on the host before any device call. Errors: IVIS_ERR_ARG for sizes, widths,
 * tolerances or option combinations out of range; IVIS_ERR_NONFINITE for a negative or
 * non-finite lambda_r / lambda_s; IVIS_ERR_OOM; IVIS_ERR_CUDA (e.g. no device). */
ivis_status ivis_plan(const ivis_config *cfg, void *stream, ivis_plan_t *out);

/* Pointing k (0 <= k < npoint): window centre at sky pixel (cx, cy) (any integers; the
 * window may extend past the sky, Eq. 2) and primary beam A_k (Eq. 3), float [nb][nb]
 * with A_k[q][p] at direction (l_p, m_q). Must be set before ivis_set_vis for k. */
ivis_status ivis_set_pointing(ivis_plan_t plan, int k, int cx, int cy, const float *beam_dev);

/* SIN re-projection of pointing k (Eq. 2; Sect. 3.3): grid_dev float [nb][nb][2] gives, for
 * each window pixel (q, p), the sampling location (X, Y) in sky pixel units (X along columns,
 * pixel centres at integers); the window becomes the bilinear interpolation of the sky there
 * (pixels off the sky count as zero; non-finite entries give zero), and the gradient its
 * transpose. Replaces the integer window of ivis_set_pointing for k; NULL restores it. The
 * gradient contributions of gridded pointings are added with atomics (not bit-reproducible). */
ivis_status ivis_set_pointing_grid(ivis_plan_t plan, int k, const float *grid_dev);

/* Host-side pre-computation of such a grid (Eq. 2; the paper's pre-processing step): window
 * pixel (q, p) of pointing k has direction cosines l = (p - nb/2) cell_rad,
 * m = (q - nb/2) cell_rad in the SIN (orthographic) frame about the pointing centre
 * (ra_k, dec_k); the same direction is projected about the sky image's reference direction
 * (ra0, dec0) with the sky image's zenithal projection sky_proj:
 *     IVIS_PROJ_SIN  (x, y) = (l', m')                         (orthographic)
 *     IVIS_PROJ_TAN  (x, y) = (l', m') / n'                    (gnomonic)
 *     IVIS_PROJ_ARC  (x, y) = (l', m') theta / sin(theta)       (zenithal equidistant,
 *                                                                theta = acos n')
 * where (l', m', n') are its direction cosines about (ra0, dec0), and lands at
 * X = crpix_x + x / cell_rad, Y = crpix_y + y / cell_rad (the same pixel size; x grows with
 * right ascension, y with declination, in both frames; angles in radians). grid_host: float
 * [nb][nb][2] (X, Y), written on the host (no device call). Directions the projection cannot
 * show (behind the tangent point for SIN and TAN, the antipode for ARC) get NaN, which the
 * gather reads as zero. With (ra_k, dec_k) = (ra0, dec0), SIN and integer crpix the grid is the
 * integer window of ivis_set_pointing centred at (crpix_x, crpix_y). Errors: IVIS_ERR_ARG for
 * nb < 1, cell_rad not finite and > 0, non-finite angles, an unknown projection or a null
 * grid. */
enum { IVIS_PROJ_SIN = 0, IVIS_PROJ_TAN = 1, IVIS_PROJ_ARC = 2 };
ivis_status ivis_reproject_grid(int nb, double cell_rad, double ra_k, double dec_k, double ra0,
                                double dec0, double crpix_x, double crpix_y, int sky_proj,
                                float *grid_host);

/* Calibrated visibilities of pair (k, chan): m points, uvw float [m][3] in wavelengths
 * (w ignored: coplanar model of Eq. 3), vis float [m][2] (re, im), weight float [m]
 * = 1/sigma^2 from the SIGMA column (Eq. 5). m == 0 declares a pair with no data;
 * 0 <= m <= 2^31 - 1025 (IVIS_ERR_ARG beyond).
 * The data are copied, converted to oversampled-grid coordinates and sorted by grid
 * tile on the device; with toeplitz = 1 the pair's Toeplitz spectrum, b window and constant
 * are computed here too. Errors: IVIS_ERR_NONFINITE for NaN/Inf or negative weights. */
ivis_status ivis_set_vis(ivis_plan_t plan, int k, int chan, int64_t m, const float *uvw_dev,
                         const float *vis_dev, const float *weight_dev);

/* Single-dish map T_b of channel chan (Eq. 12), float [n][n]; noise sigma_sd (Eq. 13)
 * and Gaussian dish beam FWHM in pixels (Eq. 11: taps truncated at +-ceil(4 sigma_B),
 * normalised to unit sum, zero outside the sky). Needed for every channel when
 * lambda_s != 0. */
ivis_status ivis_set_sd(ivis_plan_t plan, int chan, const float *tsd_dev, double sigma_sd,
                        double fwhm_pix);

/* Build work lists, allocate grids and capture the evaluation graph. Called implicitly by
 * the first evaluation; call it explicitly to keep that cost out of timed regions.
 * Errors: IVIS_ERR_STATE if a pointing, a channel's single-dish map (lambda_s != 0) or
 * every pair of a channel is missing; IVIS_ERR_ARG if more than 65535 slots (pairs with
 * visibilities, times the w-planes of a wterm plan) would be batched; IVIS_ERR_OOM. */
ivis_status ivis_prepare(ivis_plan_t plan);

/* Q_tot and its gradient at sky_dev (real [nchan][n][n]). cost_out (host) receives
 * Q_tot; terms_out (host, may be NULL) receives {Q, K, R}; grad_dev (real, same shape,
 * may alias nothing else) receives the gradient. */
ivis_status ivis_cost_grad(ivis_plan_t plan, const void *sky_dev, double *cost_out,
                           void *grad_dev, double *terms_out);

/* Asynchronous form for pipelined callers: enqueue the evaluation on the plan's stream
 * (ordered after the caller's stream) and return at once. cost_dev (device) receives
 * {Q_tot, Q, K, R}; grad_dev the gradient. Synchronise with the stream of ivis_get_stream
 * before reading either. Non-finite costs are not detected by this form. */
ivis_status ivis_cost_grad_async(ivis_plan_t plan, const void *sky_dev, void *grad_dev,
                                 double *cost_dev);

/* The plan's own CUDA stream (a cudaStream_t) on which every evaluation runs. */
ivis_status ivis_get_stream(ivis_plan_t plan, void **stream);

/* Same evaluation from HOST buffers: sky_host is copied in and the gradient copied out
 * inside the call (the end-to-end path of a host-resident caller). */
ivis_status ivis_cost_grad_host(ivis_plan_t plan, const void *sky_host, double *cost_out,
                                void *grad_host, double *terms_out);

/* Model visibilities (Eq. 3) of pair (k, chan) for sky_dev, in the caller's order of
 * ivis_set_vis: real [m][2]. */
ivis_status ivis_predict(ivis_plan_t plan, const void *sky_dev, int k, int chan,
                         void *vis_out_dev);

/* Single-dish model B (x) I (Eq. 11) of every channel: real [nchan][n][n]. Uses the
 * dish beams given by ivis_set_sd. */
ivis_status ivis_sd_predict(ivis_plan_t plan, const void *sky_dev, void *out_dev);

/* Bounded limited-memory quasi-Newton solve of Eq. 10 on the device, started from
 * sky_dev (real [nchan][n][n]; the paper starts from a null image) and overwritten with
 * the result. m_hist correction pairs (<= 32). Stops after maxiter iterations, when the
 * projected-gradient infinity norm <= pgtol, or when the relative decrease of Q_tot
 * is <= ftol. Only the cost scalar crosses to the host per evaluation. rep may be NULL. */
ivis_status ivis_solve(ivis_plan_t plan, void *sky_dev, int maxiter, int m_hist, double pgtol,
                       double ftol, ivis_solve_report *rep);

/* Same solve, also stopping as soon as Q_tot <= f_target (time-to-cost measurements, e.g. a
 * warm start against the cost a cold start reached). */
ivis_status ivis_solve_target(ivis_plan_t plan, void *sky_dev, int maxiter, int m_hist,
                              double pgtol, double ftol, double f_target, ivis_solve_report *rep);

/* Kernel width w, ES shape beta and oversampled grid size actually used. */
ivis_status ivis_get_nufft_params(ivis_plan_t plan, int *w, double *beta, int *nf);

/* Stage timing. enable != 0 re-captures the evaluation graph with CUDA event nodes around
 * every stage (on the stream each stage runs on); ivis_stage_times then fills up to cap
 * entries of names[] (static strings) and ms[] (mean milliseconds per evaluation since
 * enabling) and returns the number of stages in *count. Folding an evaluation's events into
 * the totals synchronises the plan's stream before the next evaluation starts. */
ivis_status ivis_profile(ivis_plan_t plan, int enable);
ivis_status ivis_stage_times(ivis_plan_t plan, const char **names, double *ms, int cap,
                             int *count);

/* Tuning in use: max visibilities per grid-pass chunk, columns per CTA of the column FFT
 * passes, and a text record of the autotuner's decision (empty when not tuned). */
ivis_status ivis_tuning(ivis_plan_t plan, int *chunk_cap, int *fft_cols, const char **text);

/* Number of kernel launches one evaluation issues (the graph's kernel nodes). */
ivis_status ivis_launches_per_eval(ivis_plan_t plan, int *count);

/* Allocation-free single-dish model B (x) I, for callers that cannot allocate device memory
 * when they need it (e.g. inside a region whose memory a pool or an outside framework owns,
 * or an embedded host that forbids runtime allocation). No counterpart in the paper: it is
 * the same separable dish-beam convolution as ivis_sd_predict (Gaussian taps truncated at
 * +-ceil(4 sigma), unit sum, zero outside the image), computed without a plan and without
 * allocating: its scratch (taps and the row-pass image of one channel) lives in a
 * file-scope device array of about 4 MiB (1632 + 1,048,576 floats) that every GPU loading the
 * library keeps until the process exits. sky_dev, out_dev: float [nchan][n][n] on the current
 * device; stream: a cudaStream_t (NULL = legacy default stream). The call is synchronous: it
 * copies the taps from host memory and returns after the work completes, so it cannot be
 * recorded into a CUDA graph; on a stream that is capturing it returns IVIS_ERR_STATE without
 * touching the stream. Limits: n * n <= 1,048,576 and ceil(4 sigma) <= 812 (FWHM <= 478
 * pixels), else IVIS_ERR_ARG with a message. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress). Every call shares the one array: calls that overlap
 * on the GPU (other streams, other host threads) race and must be serialised by the caller.
 * Calls no cudaMalloc/cudaFree. Errors are reported by ivis_last_error(NULL). */
ivis_status ivis_sd_predict_noalloc(const float *sky_dev, int n, int nchan, double fwhm_pix,
                                    float *out_dev, void *stream);

/* Inputs of the learned warm start (an extension; not in the paper): the dirty
 * image -grad Q(0) of each channel (the adjoint of the weighted data, Eqs. 5-6 at I = 0;
 * real [nchan][n][n] on the device) and, if beamw_dev is not NULL, the beam-weight map
 * sum_k A_k^2 of the linear mosaic of Sect. 4.3 (real [n][n]). */
ivis_status ivis_dirty_image(ivis_plan_t plan, void *dirty_dev, void *beamw_dev);

/* Short-spacing correction by feathering (the paper's appendix; a post-processing step of the
 * reconstructed cube): per channel, on the plan's n x n grid with no padding,
 *     out = IDFT[ B DFT(sd_scale * sd) + (1 - B) DFT(int) ],
 *     B(k) = exp(-2 pi^2 sigma^2 |k|^2),  sigma = theta / (2 sqrt(2 ln 2)),
 * with k in cycles per radian (theta_rad in radians; pixels of the plan's cell_rad); the real
 * part is returned. int_dev and out_dev: real [nchan][n][n] in the plan's precision (out must
 * not alias int); sd_dev: float [nchan][n][n], the single-dish map regridded onto the image
 * grid, multiplied by sd_scale (e.g. ivis_rayleigh_jeans(nu) for maps in kelvin). Needs n a
 * power of two in [16, 4096]. Errors: IVIS_ERR_ARG. Runs on the plan's stream; returns after
 * the result is written. */
ivis_status ivis_feather(ivis_plan_t plan, const void *int_dev, const float *sd_dev, double theta_rad,
                         double sd_scale, void *out_dev);

/* Rayleigh-Jeans conversion of the same appendix: Jy per square arcsecond per kelvin of
 * brightness temperature at frequency freq_hz, 2 k nu^2 / c^2 (SI constants). */
double ivis_rayleigh_jeans(double freq_hz);

/* ---- learned warm start: a 4-level U-Net [dirty image, beam-weight map] -> initial sky ----
 * No counterpart in the paper (its closest hook is the "physically motivated priors" of its
 * future prospects). Per level two 3x3 convolutions + ReLU; encoder widths c, 2c, 4c, 8c with
 * 2x2 max pooling; decoder: nearest 2x upsampling, concatenation with the encoder output of
 * the same level, two 3x3 convolutions + ReLU; a 1x1 head; loss = mean squared error.
 * BF16 weights and activations, FP32 accumulation and gradients, FP32 Adam.
 * Parameters are one flat float vector: for each 3x3 layer in order (enc 0a, 0b, 1a, 1b, 2a,
 * 2b, 3a, 3b, dec 2a, 2b, 1a, 1b, 0a, 0b) the weights W[cout][tap = 3 dy + dx][cin] then the
 * bias[cout]; then the head weights [c] and bias [1]. Decoder "a" layers take the upsampled
 * deeper tensor's channels first, then the skip channels. */
typedef struct ivis_unet_s *ivis_unet_t;

/* Create a network of base width c (multiple of 8, 8..64) for batches up to max_batch images
 * of up to max_hw pixels; work runs on stream (cudaStream_t; NULL = legacy default). The
 * parameters start at zero: set them with ivis_unet_set_params. */
ivis_status ivis_unet_create(int base_channels, int max_batch, int max_hw, void *stream,
                             ivis_unet_t *out);
ivis_status ivis_unet_num_params(ivis_unet_t net, int64_t *n);
/* Copy the flat parameter vector from / to host memory (float [n]); set also resets Adam. */
ivis_status ivis_unet_set_params(ivis_unet_t net, const float *host_params);
ivis_status ivis_unet_get_params(ivis_unet_t net, float *host_params);
/* Forward: in_dev float [B][2][H][W] (plane 0 dirty image, plane 1 beam-weight map), out_dev
 * float [B][H][W]; H and W multiples of 8. */
ivis_status ivis_unet_forward(ivis_unet_t net, const float *in_dev, float *out_dev, int B, int H,
                              int W);
/* The warm start of one channel, straight from the solver's planes: dirty_dev and beamw_dev
 * (the planes ivis_dirty_image writes; [H][W], double if fp64 else float) become the network
 * input (s0 dirty, s1 beam weight) and x0_dev ([H][W], same type) receives
 * max(s_out * U-Net(input), 0), the initial sky for ivis_solve. One image (B = 1), H and W
 * as for ivis_unet_forward. Runs on the network's stream and returns after it; inputs must be
 * complete on that stream. Scales must be finite. */
ivis_status ivis_unet_warm_start(ivis_unet_t net, const void *dirty_dev, const void *beamw_dev,
                                 int fp64, int H, int W, double s0, double s1, double s_out,
                                 void *x0_dev);
/* Training tensors from the solver's planes: out_dev (float) gets sa * a in its first npix
 * entries and, when b_dev is not NULL, sb * b in the next npix (a network input [2][H][W]);
 * a and b are double if fp64 else float; products are taken in that type. Queued on stream
 * (cudaStream_t; NULL = legacy default); does not wait. Errors: ivis_unet_last_error(NULL). */
ivis_status ivis_unet_planes(const void *a_dev, const void *b_dev, int fp64, int64_t npix,
                             double sa, double sb, float *out_dev, void *stream);
/* Forward + backward of the MSE loss against tgt_dev (float [B][H][W]); the parameter
 * gradient (zeroed first) stays on the device; loss_out (host, may be NULL) gets the loss. */
ivis_status ivis_unet_backward(ivis_unet_t net, const float *in_dev, const float *tgt_dev, int B,
                               int H, int W, double *loss_out);
ivis_status ivis_unet_get_grads(ivis_unet_t net, float *host_grads);
/* One Adam update with the last gradient (Kingma & Ba 2015, bias-corrected). */
ivis_status ivis_unet_adam_step(ivis_unet_t net, float lr, float beta1, float beta2, float eps);
/* Forward convolutions and the parameter-gradient GEMMs of the backward on the 5th-generation
 * tensor cores (tcgen05.mma, accumulators in tensor memory; default), or all GEMMs on mma.sync
 * (enable = 0). The activation-gradient GEMMs use mma.sync in both modes. A tensor-core
 * completion wait that runs out returns IVIS_ERR_TIMEOUT. */
ivis_status ivis_unet_use_tcgen05(ivis_unet_t net, int enable);
ivis_status ivis_unet_destroy(ivis_unet_t net);
const char *ivis_unet_last_error(ivis_unet_t net);

/* Release every device resource of the plan. Safe on NULL. */
ivis_status ivis_destroy(ivis_plan_t plan);

/* Text of the last error on this plan (or of the last failed ivis_plan when plan is
 * NULL). Valid until the next call on the plan. */
const char *ivis_last_error(ivis_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* IVIS_H */
