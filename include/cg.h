/*
 * cg.h -- C ABI of libcg: objective values and exact reverse-mode gradients
 * of histogram and event fit objectives, computed by hand-written sm_103a
 * CUDA kernels.
 *
 * The problem is the one of the paper's histogram-fitting use of AD
 * (Sec. 4, Fig. 3): a parameter vector and data go in, the objective value
 * and its exact gradient with respect to the parameters come out.  The
 * gradient is the reverse-mode (adjoint) derivative of Sec. 1-2: one fused
 * pass evaluates each bin's or event's term and sweeps its adjoint back to
 * the parameters, and the per-element parameter adjoints are summed -- the
 * "parallel reads become parallel writes" situation of Sec. 3, handled here
 * by a deterministic reduction (warp shuffle, then block, then a fixed-order
 * sum over blocks) with no floating-point atomics.
 *
 * Conventions for every call:
 *  - Pointers documented "device" are caller-owned device memory; the
 *    library never allocates or frees device memory.  Scratch comes from a
 *    caller-provided workspace `ws` of at least the size the matching
 *    *_workspace_size() call returns (256-byte aligned).
 *  - Structs (cg_problem, cg_batch, cg_tile_map) are host memory read during
 *    the call only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on it and may be captured in a CUDA
 *    graph; argument errors are returned synchronously before any launch.
 *  - Device-detected problems (log of a non-positive model value, a
 *    non-finite parameter, a wait that ran out) do not stop the kernels;
 *    they are recorded in a status word inside `ws`, read by cg_get_status().
 *  - All results are deterministic for a given launch configuration: the
 *    summation tree depends on the problem size and the tile mapping only.
 *  - No call throws, traps or asserts on the device.
 */
#ifndef CG_H
#define CG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CG_OK = 0,
    CG_ERR_INVALID_ARG = 1,  /* bad sizes, null pointers, unknown enums */
    CG_ERR_DOMAIN = 2,       /* device: log of a non-positive model value or non-finite term */
    CG_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
    CG_ERR_TIMEOUT = 4,      /* device: a bounded wait gave up */
    CG_ERR_NOT_CONVERGED = 5,
    CG_ERR_UNSUPPORTED = 6,  /* combination not implemented */
    CG_ERR_WORKSPACE = 7     /* workspace missing, misaligned or too small */
} cg_status;

/* Model families (parameter order is fixed and part of the ABI):
 *  CG_MODEL_GAUSS_POLY   1-D binned: K Gaussian peaks (amplitude = peak
 *                        height, the "gaus" of Fig. 3a) plus a polynomial of
 *                        degree D: theta = (A_1, mu_1, s_1, ..., A_K, mu_K,
 *                        s_K, c_0, ..., c_D), P = 3K + D + 1.
 *                        f(x) = sum_k A_k exp(-(x-mu_k)^2/(2 s_k^2)) + sum_j c_j u^j
 *                        with u = x (poly_mode 0) or u = (2x-lo-hi)/(hi-lo) (1).
 *  CG_MODEL_MIX_GAUSS_EXP unbinned on [lo, hi]: theta = (frac, mu, s, lambda),
 *                        p(x) = frac N(x;mu,s)/Z_G + (1-frac) lambda e^{-lambda x}/Z_E,
 *                        each component normalised over [lo, hi].
 *  CG_MODEL_ROTGAUSS2D   2-D binned: K rotated Gaussians + constant:
 *                        theta = (A, mu_x, mu_y, s_x, s_y, phi) x K, then C.
 */
typedef enum {
    CG_MODEL_GAUSS_POLY = 0,
    CG_MODEL_MIX_GAUSS_EXP = 1,
    CG_MODEL_ROTGAUSS2D = 2
} cg_model;

/* Objectives (the per-element term T_i; the objective is sum_i T_i):
 *  CG_OBJ_CHI2        w_i (y_i - f_i)^2, w_i = 1/max(y_i, 1)
 *  CG_OBJ_POISSON     f_i - y_i log f_i              (log y_i! dropped)
 *  CG_OBJ_POISSON_BC  2 (f_i - y_i + y_i log(y_i/f_i)), 2 f_i when y_i = 0
 *  CG_OBJ_UNBINNED_NLL -w_i log p(x_i)               (w_i = 1 without weights)
 */
typedef enum {
    CG_OBJ_CHI2 = 0,
    CG_OBJ_POISSON = 1,
    CG_OBJ_POISSON_BC = 2,
    CG_OBJ_UNBINNED_NLL = 3
} cg_objective_kind;

/* Arithmetic of the per-element work.  Accumulation is FP64 in every mode.
 *  CG_PREC_FP64  FP64 throughout (the FP64 pipe).
 *  CG_PREC_DF64  per-element arithmetic in double-float (pairs of FP32
 *                values with error-free transformations) on the FP32 pipe;
 *                per-term relative error about 1e-14, stated per workload
 *                by the test suite against FP64. */
typedef enum {
    CG_PREC_FP64 = 0,
    CG_PREC_DF64 = 1
} cg_precision;

#define CG_MAX_PEAKS_1D 4
#define CG_MAX_POLY_DEGREE 3
#define CG_MAX_PEAKS_2D 8
#define CG_MAX_PARAMS 49

/* One fit problem: model, objective and data (host struct). */
typedef struct {
    int32_t model;          /* cg_model */
    int32_t objective;      /* cg_objective_kind */
    int32_t precision;      /* cg_precision */
    int32_t n_peaks;        /* K: 0..CG_MAX_PEAKS_1D (1-D), 1..CG_MAX_PEAKS_2D (2-D) */
    int32_t poly_degree;    /* D: -1..CG_MAX_POLY_DEGREE (1-D only) */
    int32_t poly_mode;      /* 0: powers of x, 1: powers of t = (2x-lo-hi)/(hi-lo) */
    int64_t n_bins[2];      /* binned: bins along x and y (1-D uses n_bins[0]) */
    double lo[2], hi[2];    /* range along x and y; bin centres are lo+(i+0.5)(hi-lo)/n */
    const double *centres;  /* device, optional explicit 1-D bin centres [n_bins[0]] (NULL: uniform) */
    const double *data;     /* device: counts, 1-D [n_bins[0]] or 2-D [n_bins[1]][n_bins[0]]
                               (x index fastest); unbinned: events [n_events] */
    const double *weights;  /* device, optional per-event weights [n_events] (unbinned only) */
    int64_t n_events;       /* unbinned: number of events */
} cg_problem;

/* Many histograms of one model/objective, concatenated (host struct).
 * Histogram h owns bins offsets[h] .. offsets[h+1]-1 of tmpl.data and has
 * range [lo[h], hi[h]] with uniform bins.  When offsets == NULL the batch is
 * n_hist parameter points on the single problem `tmpl`. */
typedef struct {
    cg_problem tmpl;
    int64_t n_hist;
    const int64_t *offsets; /* device [n_hist + 1], or NULL */
    const double *lo;       /* device [n_hist], used when offsets != NULL */
    const double *hi;       /* device [n_hist], used when offsets != NULL */
} cg_batch;

/* Number of parameters P of the problem's model, or -1 if it is invalid. */
int cg_num_params(const cg_problem *pb);

/* Workspace bytes for cg_objective / cg_gradient (n_theta = 1) and
 * cg_batch_gradient with offsets == NULL (n_theta = n_hist).  0 when the
 * problem is invalid. */
size_t cg_workspace_size(const cg_problem *pb, int64_t n_theta);

/* Objective value at one parameter point (Sec. 4: the fit objective).
 * theta: device [P]; value: device [1].  Runs the same fused kernel as
 * cg_gradient and discards the gradient. */
cg_status cg_objective(const cg_problem *pb, const double *theta, double *value,
                       void *ws, size_t ws_bytes, void *stream);

/* Objective value and its exact gradient at one parameter point: the fused
 * per-element forward evaluation + adjoint sweep (reverse mode, Sec. 1-2;
 * the generated-gradient-in-a-kernel pattern of Listing 1, here with the
 * per-parameter adjoints reduced over all elements as Sec. 3 requires).
 * theta: device [P]; value: device [1]; grad: device [P]. */
cg_status cg_gradient(const cg_problem *pb, const double *theta, double *value, double *grad,
                      void *ws, size_t ws_bytes, void *stream);

/* Values and gradients for many parameter points or many histograms in one
 * launch sequence.  theta: device [n_hist][P] (row-major); value: device
 * [n_hist]; grad: device [n_hist][P].
 *  - offsets == NULL: n_hist parameter points on the single problem tmpl
 *    (one thread per evaluation in Listing 1; here each point's gradient is
 *    itself a reduction over all bins or events).  grad may be NULL: values
 *    only (value-only kernels for the 1-D model in CG_PREC_DF64).
 *  - offsets != NULL: histogram h is evaluated at theta[h]; binned 1-D
 *    models only; grad may be NULL: values only (no adjoint sweep).
 *    Workspace: cg_batch_workspace_size(). */
size_t cg_batch_workspace_size(const cg_batch *b);
cg_status cg_batch_gradient(const cg_batch *b, const double *theta, double *value, double *grad,
                            void *ws, size_t ws_bytes, void *stream);

/* Device status recorded by the last call that used `ws`: synchronises
 * `stream`, returns CG_OK, CG_ERR_DOMAIN or CG_ERR_TIMEOUT (or CG_ERR_CUDA
 * if the copy fails). */
cg_status cg_get_status(const void *ws, void *stream);

/* ------------------------------------------------------------------------
 * Gradient without any caller-provided or library-allocated device memory.
 * The paper has no counterpart; this exists for callers that cannot
 * allocate device memory or pass a workspace (code running under another
 * framework's allocator or memory pool, plug-ins whose host owns every
 * device buffer, real-time loops where an allocation may block or fail).
 *
 * Same result as cg_batch_gradient with offsets == NULL for the unbinned
 * mixture model (CG_MODEL_MIX_GAUSS_EXP, CG_OBJ_UNBINNED_NLL, CG_PREC_FP64),
 * for n_theta parameter points: theta device [n_theta][4], value device
 * [n_theta], grad device [n_theta][4]; events (and optional weights) as in
 * cg_problem.  The per-tile partial sums live in one static device array of
 * CG_NOALLOC_SCRATCH_BYTES bytes inside libcg, created on every GPU that
 * loads the library and kept until the process exits.
 *  - n_theta > CG_NOALLOC_MAX_POINTS returns CG_ERR_INVALID_ARG (the array
 *    would not hold the partials); so do other models or precisions.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before capturing any stream.
 *  - It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - All calls share the array and it keeps the last call's contents; every
 *    call overwrites the slots it reads, so nothing is cleared.  Calls that
 *    overlap on the GPU (other streams, other host threads) race on it.
 *  - A parameter point whose terms hit a domain error gets a NaN value
 *    (there is no workspace status word to read). */
#define CG_NOALLOC_SCRATCH_BYTES (1u << 20)
#define CG_NOALLOC_MAX_POINTS 4096
cg_status cg_mixture_gradient_noalloc(const cg_problem *pb, const double *theta, int64_t n_theta,
                                      double *value, double *grad, void *stream);

/* ------------------------------------------------------------------------
 * Learned start (a network that proposes fit starting parameters).  The
 * paper has no network; these calls serve the BF16 multilayer perceptron
 * that maps a coarse rebinned histogram to starting parameters, trained and
 * run by the kernels below.
 * ------------------------------------------------------------------------ */

/* C[M][N] = sum_k A(m, k) B(n, k) on the tensor cores: BF16 operands
 * (uint16 storage), FP32 accumulation in tensor memory.  A is [M][lda]
 * (transA = 0) or [K][lda] read transposed (transA = 1); B is [N][ldb]
 * (transB = 0) or [K][ldb] (transB = 1); C row stride ldc.  Epilogues:
 * 0 Cf = acc; 1 Cf = acc + bias[n]; 2 z = acc + bias[n], aux_out = z,
 * Cb = bf16(gelu(z)) (and Cf = gelu(z) if given); 3 dz = acc * gelu'(aux_in),
 * Cb = bf16(dz) (and/or Cf = dz).  gelu(z) = z Phi(z).  err (device int, may
 * be NULL) gets bit 0 when a bounded wait on the tensor core gave up.
 * Kernels: K-major operands (transA = transB = 0) with lda, ldb multiples of
 * 8 and 16-byte aligned A, B go through TMA loads (128-byte swizzle) into an
 * mbarrier ring feeding tcgen05.mma: for N >= 128 a persistent kernel (one
 * CTA per SM, 128 x 256 or 128 x 128 tiles, two TMEM accumulators so that a
 * tile's epilogue overlaps the next tile's MMAs), for smaller N one CTA per
 * tile; other operands are staged through registers.  Results do not depend
 * on the kernel chosen beyond FP32 rounding of the accumulation order. */
cg_status cg_gemm_bf16(const void *A, const void *B, int M, int N, int K, int lda, int ldb, int transA,
                       int transB, float *Cf, void *Cb, int ldc, const float *bias, const float *aux_in,
                       float *aux_out, int epilogue, int *err, void *stream);

/* Failure detection (not in the paper): every wait of the kernels above on
 * another role or on the tensor core is bounded (about 1 s) and, when it
 * gives up, sets bit 0 of `err` and lets the kernel end with nothing in
 * flight.  This call runs that wait on a barrier that nothing completes, so
 * that a test can see the limit work: after about 1 s bit 0 of *err (device
 * int) is set; the context stays usable.  CG_ERR_INVALID_ARG for a NULL err. */
cg_status cg_check_wait_timeout(int *err, void *stream);

/* Rebinning for the network input: x[h][j] = bf16(r_j / max_j r_j) with
 * r_j the sum of `factor` consecutive counts of histogram h (y: device
 * [H][n_bins] FP64, x: device [H][n_bins/factor] bf16); scale[h] = max_j r_j. */
cg_status cg_rebin_normalize(const double *y, int64_t H, int n_bins, int factor, void *x_bf16, float *scale,
                             void *stream);

/* Plain heuristic starting point for K Gaussian peaks + linear background on
 * [lo, hi] (y: device [H][n_bins] FP64; theta0: device [H][3K+2]): on the
 * histogram rebinned by `factor` (sums in bin order), 5-bin box smoothing,
 * background line through the minima (first index of each) of the first and
 * last eighth, the K highest local maxima of the residual (first index on
 * ties), each at least 3 rebinned bins from every earlier one, width from the
 * half-maximum crossings; peaks sorted by position.  Products and sums are
 * rounded separately (no fused multiply-add), so the result is reproducible
 * bit for bit.  K <= 8, n_bins/factor in [8, 3072]. */
cg_status cg_heuristic_start(const double *y, int64_t H, int n_bins, int factor, double lo, double hi, int n_peaks,
                             double *theta0, void *stream);

/* Refinement of starting points of K peaks + linear background on the
 * full-resolution histogram (y: device [H][n_bins] FP64 on [lo, hi];
 * theta_in / theta_out: device [H][3K+2], (A, mu, s) per peak then b0, b1;
 * theta_out may equal theta_in).  Not in the paper: it sharpens a coarse
 * start (the network's proposal from the rebinned histogram, or the
 * heuristic's) before the fit.  One warp per histogram, `sweeps` passes over
 * the peaks in order of position: for peak k the counts within
 * mu_k +- w_k, w_k = half_width max(s_k, 4 h) (h the bin width), less the
 * background and the other peaks at the current parameters, are clipped
 * at zero and give moments S0, S1, S2 about mu_k; then mu_k += S1/S0, the
 * width is the one whose Gaussian truncated at +-w_k has the variance
 * S2/S0 - (S1/S0)^2 (one fixed-point step of var = s^2 (1 - 2 z phi(z) /
 * erf(z/sqrt 2)), z = w/s, z clamped to [0.5, 10]), and the height makes
 * the truncated Gaussian's sum S0.  A peak whose window holds no positive
 * residual keeps its parameters; peaks leave sorted by position.  FP64;
 * window bounds and centres rounded operation by operation (no fused
 * multiply-add).  K <= 8, sweeps in [0, 16], half_width in (0, 10]. */
cg_status cg_refine_start(const double *y, int64_t H, int n_bins, double lo, double hi, int n_peaks,
                          const double *theta_in, double *theta_out, int sweeps, double half_width, void *stream);

/* loss = mean over B x n_out of (pred - target)^2 (pred rows of stride ld,
 * target [B][n_out]); dpred (FP32) and/or dpred_bf16 get its gradient, zero in
 * the padding columns.  One CTA, fixed-order sums. */
cg_status cg_mse_loss(const float *pred, const float *target, int64_t B, int n_out, int ld, float *loss,
                      float *dpred, void *dpred_bf16, void *stream);

/* out[c] = sum over rows of X[r][c] (X: [rows][cols] FP32), rows in order. */
cg_status cg_colsum(const float *X, int64_t rows, int cols, float *out, void *stream);

/* One AdamW step on FP32 master weights w (n values) with moments m, v;
 * bias-corrected with `step` (>= 1); w_bf16 (optional) receives the rounded
 * copy used by the GEMMs. */
cg_status cg_adamw(float *w, const float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2,
                   float eps, float weight_decay, int step, void *w_bf16, void *stream);

/* Network output -> starting parameters of K peaks + linear background:
 * y rows (stride ld) hold z-scores (mean, stdv: [3K+2]) of
 * (A_k factor/scale, mu_k, log s_k, b0 factor/scale, b1 factor/scale);
 * the decoded values are clamped into the model's domain and the peaks are
 * sorted by mu.  theta0: device [H][3K+2] FP64. */
cg_status cg_decode_start(const float *y, int ld, const float *scale, const float *mean, const float *stdv,
                          int64_t H, int n_peaks, int factor, int n_bins, double lo, double hi, double *theta0,
                          void *stream);

/* Per histogram h, theta_out[h] = theta_a[h] if fa[h] <= fb[h] (a non-finite
 * value loses), else theta_b[h]: the objective judges two candidate starts.
 * took_a (optional, device [H]) records the choice. */
cg_status cg_select_start(const double *fa, const double *fb, const double *theta_a, const double *theta_b,
                          int64_t H, int P, double *theta_out, int *took_a, void *stream);

/* b[i] = bf16(a[i]). */
cg_status cg_to_bf16(const float *a, int64_t n, void *b, void *stream);

/* Profiling hook: when start/stop are non-NULL cudaEvent_t handles (passed as
 * void*), every later launch of a fused accumulation kernel (the dominant
 * kernel of cg_objective / cg_gradient / cg_batch_gradient / cg_fit_*)
 * records `start` immediately before and `stop` immediately after it, on the
 * call's stream.  NULL, NULL switches it off.  Process-wide; not meant to be
 * changed while other threads are calling the library. */
void cg_set_profile_events(void *start, void *stop);

/* Static description of a status code. */
const char *cg_status_string(cg_status s);

/* ------------------------------------------------------------------------
 * Fitting (Sec. 4: AD gradients replacing numerical ones inside the
 * histogram fitter; the minimiser is gradient-only since second
 * derivatives are not taken from AD).  The minimiser is BFGS with a
 * backtracking Armijo line search; see cg_fit_step.
 * ------------------------------------------------------------------------ */

#define CG_FIT_MAX_PARAMS 12

enum {
    CG_FIT_RUNNING = 0,
    CG_FIT_CONVERGED = 1,
    CG_FIT_MAX_ITER = 2,
    CG_FIT_LINESEARCH_FAILED = 3,
    CG_FIT_DOMAIN = 4
};

/* Per-histogram fit state (device memory, one per histogram). */
typedef struct {
    double theta[CG_FIT_MAX_PARAMS];
    double grad[CG_FIT_MAX_PARAMS];
    double hinv[CG_FIT_MAX_PARAMS * CG_FIT_MAX_PARAMS]; /* inverse-Hessian approximation, row-major P x P */
    double h0[CG_FIT_MAX_PARAMS];   /* initial diagonal: 1 / Gauss-Newton diagonal */
    double f;                       /* objective at theta */
    double edm;                     /* g^T H g / 2 */
    double fdata;                   /* the part of f that depends on the counts alone (Baker-Cousins:
                                       2 sum (y log y - y) over y > 0; chi2, Poisson: 0), written by
                                       the FP64 init calls; cg_fit_step's FP64 evaluations skip that
                                       part per bin and add this sum instead.  0 after a df64 or
                                       Levenberg-Marquardt init, whose evaluations include it. */
    int32_t iter;                   /* accepted iterations */
    int32_t n_eval;                 /* objective+gradient evaluations */
    int32_t status;                 /* CG_FIT_* */
    int32_t n_params;
} cg_fit_state;

/* How histograms are mapped onto the GPU by the batched fitter.  Histograms
 * with n <= warp_max_bins are fitted by one warp each, those with
 * n <= cta_max_bins by one CTA each, larger ones by a cluster of
 * cluster_size CTAs.  Chosen by the autotuner in the Python layer. */
typedef struct {
    int32_t warp_max_bins;
    int32_t cta_max_bins;
    int32_t cta_threads;     /* 64..512, multiple of 32 */
    int32_t cluster_size;    /* 1, 2, 4 or 8 */
} cg_tile_map;

/* Workspace for the batched fit calls on batch b (offsets != NULL): header,
 * work queues and per-histogram scratch. */
size_t cg_fit_workspace_size(const cg_batch *b);

/* Work queues of the batched fitter, built on the host from the host copy of
 * the bin offsets (host_offsets[n_hist + 1]): histograms with more than
 * map->cta_max_bins bins go to the cluster queue (or the CTA queue when
 * cluster_size == 1), those with more than map->warp_max_bins to the CTA
 * queue, the rest to the warp queue; each queue is sorted by decreasing
 * size.  Also stores every histogram by decreasing size, the order in which
 * cg_fit_init's evaluation kernel takes them (one CTA per histogram from an
 * atomic counter).  Uploaded into ws; this call synchronises `stream`.  Must
 * precede cg_fit_init / cg_fit_step on the same ws with the same map. */
cg_status cg_fit_plan(const cg_batch *b, const int64_t *host_offsets, const cg_tile_map *map,
                      void *ws, size_t ws_bytes, void *stream);

/* Initialise fit states at theta0 (device [n_hist][P], P <= CG_FIT_MAX_PARAMS):
 * one evaluation of F, g and the Gauss-Newton diagonal GN per histogram,
 * H = diag(1/GN) (1 where GN <= 0), status CG_FIT_RUNNING, or CG_FIT_DOMAIN
 * when F(theta0) is not finite.  Binned 1-D models with 1..3 peaks. */
cg_status cg_fit_init(const cg_batch *b, const cg_tile_map *map, const double *theta0,
                      cg_fit_state *state, void *ws, size_t ws_bytes, void *stream);

/* Run up to n_steps BFGS iterations on every histogram whose status is
 * CG_FIT_RUNNING, in ONE persistent launch (after a 16-byte reset of the
 * queue counters): warps, CTAs and CTA clusters pop histograms from their
 * queues.  One iteration: d = -H g (reset to the initial diagonal when
 * g.d >= 0); trial points theta + alpha d from alpha = 1, accepted when
 * F(trial) <= F + 1e-4 alpha g.d, otherwise alpha becomes the minimiser of
 * the quadratic through F, g.d and F(trial) clamped to [0.1, 0.5] alpha
 * (0.1 alpha for a non-finite F), at most 20 trials (then
 * CG_FIT_LINESEARCH_FAILED); BFGS update when s.y > 1e-12 |s||y|;
 * CG_FIT_CONVERGED when EDM = g.H.g/2 < tol max(1, |F|) (also checked
 * before the first iteration).  Capturable in a CUDA graph. */
cg_status cg_fit_step(const cg_batch *b, const cg_tile_map *map, cg_fit_state *state, int n_steps,
                      double tol, void *ws, size_t ws_bytes, void *stream);

/* Gauss-Newton matrix of a batched binned fit (df64 batches only, else
 * CG_ERR_UNSUPPORTED): for every histogram h, value[h], grad[h][P] and
 * gn[h][P][P] (row-major, symmetric) at theta[h][P], with P = 3 n_peaks +
 * poly_degree + 1.  GN = sum over bins of T''(f) (df/dtheta)(df/dtheta)^T,
 * the Hessian of the objective with the model's own curvature dropped (the
 * second derivatives Sec. 4 says the minimiser still takes by finite
 * differences, here from the same reverse sweep); T'' = 2/max(y,1)
 * for chi2, y/f^2 for Poisson, 2 y/f^2 for Baker-Cousins.  The products are
 * accumulated in FP32: with m bins per thread an entry is within about
 * (m + 8) 2^-24 sqrt(GN_aa GN_bb) (1e-5 at 20,000 bins); the value and
 * gradient are the df64 ones.  value[h] is NaN where the model
 * leaves its domain or the histogram has 2^24 bins or more.  ws: >= 256
 * bytes, 256-byte aligned (unused; reserved). */
cg_status cg_batch_gn(const cg_batch *b, const double *theta, double *value, double *grad, double *gn,
                      void *ws, size_t ws_bytes, void *stream);

/* Levenberg-Marquardt fits of every histogram of a df64 batch, a second-order
 * alternative to cg_fit_step: each step evaluates value, gradient and the
 * Gauss-Newton matrix at the trial points (tiled, below) and runs the control,
 * one warp per histogram.  A trial is
 * accepted when F(trial) < F; then lambda /= 10 (floor 1e-12), otherwise
 * lambda *= 10 (CG_FIT_LINESEARCH_FAILED past 1e16); the next trial is
 * theta + delta with (GN + lambda diag(GN)) delta = -g solved by Cholesky
 * (diagonal entries <= 0 count as 1; a scaled gradient step where the matrix
 * is not positive definite).  CG_FIT_CONVERGED when EDM = g^T GN^-1 g / 2 <
 * tol max(1, |F|), GN the undamped matrix at theta.  state[h].hinv holds GN
 * (not an inverse), h0[0] lambda; iter counts accepted steps, n_eval
 * evaluations; a fit that has not converged after the last step keeps
 * CG_FIT_RUNNING (more steps continue it).  init evaluates theta0
 * [n_hist][P] (device) and sets lambda = 1e-3.  Capturable in a CUDA graph.
 * Evaluation: the plan cuts every histogram into tiles of at most 16384 bins
 * (histograms by decreasing size); per step, CTAs take tiles from a counter
 * and write one partial row per tile (df64 value and gradient sums, a domain
 * flag, FP32 Gauss-Newton products), then one warp per histogram sums its
 * rows in tile order and runs the control.  Results do not depend on which
 * CTA took which tile.
 * ws: cg_fit_lm_workspace_size bytes, 256-byte aligned, written by
 * cg_fit_lm_plan (host offsets host_offsets[n_hist + 1]; synchronises
 * `stream`) before init / step.  A workspace without a plan makes init and
 * step do nothing (the kernels check the plan's header and tile count
 * against ws_bytes).  Histograms of 2^24 bins or more end CG_FIT_DOMAIN. */
size_t cg_fit_lm_workspace_size(const cg_batch *b, const int64_t *host_offsets);
cg_status cg_fit_lm_plan(const cg_batch *b, const int64_t *host_offsets, void *ws, size_t ws_bytes,
                         void *stream);
cg_status cg_fit_lm_init(const cg_batch *b, const double *theta0, cg_fit_state *state, double tol, void *ws,
                         size_t ws_bytes, void *stream);
cg_status cg_fit_lm_step(const cg_batch *b, cg_fit_state *state, int n_steps, double tol, void *ws,
                         size_t ws_bytes, void *stream);

/* The same iteration for ONE histogram on the full GPU (the plain
 * per-histogram path): every trial point is one cg_gradient-style launch
 * pair (tile kernel + finalize) followed by a one-warp control kernel; no
 * host synchronisation.  Once the fit stops, later launches of the call
 * return immediately.  state: device [1]. */
size_t cg_fit_single_workspace_size(const cg_problem *pb);
cg_status cg_fit_single_init(const cg_problem *pb, const double *theta0, cg_fit_state *state,
                             void *ws, size_t ws_bytes, void *stream);
cg_status cg_fit_single_step(const cg_problem *pb, cg_fit_state *state, int n_evals, double tol,
                             void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Expression programs: the per-element term of an objective written as an
 * expression, differentiated by source transformation.  The paper's tool
 * turns the source of a C++ function into the source of its reverse-mode
 * derivative (Sec. 2-3, Listings 1-2); here the function is a small
 * expression DAG and libcg writes the CUDA source of one fused kernel (the
 * forward evaluation and the reverse sweep of every element, summed per
 * tile in a fixed order) plus a finalize kernel (chunk-ordered sums and the
 * reverse sweep of the parameter-only part), compiles it at run time with
 * NVRTC for this GPU and launches it.  Objective = sum over the n elements
 * of the root node; gradient with respect to the parameters.
 *
 * Nodes are given in topological order (operands a, b refer to earlier
 * nodes); the last node is the per-element term.  Subexpressions of the
 * parameters alone (normalisations, 1/(2 s^2)) are evaluated once per
 * parameter point and their adjoints accumulated over the elements, then
 * chained to the parameters once (the prologue / epilogue of the hand-written
 * kernels).  FP64 throughout.
 * ------------------------------------------------------------------------ */
typedef enum {
    CG_EX_CONST = 0,   /* the constant c */
    CG_EX_PARAM = 1,   /* theta[i] */
    CG_EX_INPUT = 2,   /* input array i at the element */
    CG_EX_INDEX = 3,   /* the element index, as a double */
    CG_EX_ADD = 4,     /* a + b */
    CG_EX_SUB = 5,     /* a - b */
    CG_EX_MUL = 6,     /* a * b */
    CG_EX_DIV = 7,     /* a / b */
    CG_EX_NEG = 8,     /* -a */
    CG_EX_EXP = 9,     /* exp(a) */
    CG_EX_LOG = 10,    /* log(a) */
    CG_EX_SQRT = 11,   /* sqrt(a) */
    CG_EX_ERFC = 12,   /* erfc(a) */
    CG_EX_POWI = 13,   /* a^i, integer i in [-16, 16] */
    CG_EX_MAX = 14     /* max(a, b); the derivative goes to a when a >= b */
} cg_expr_op;

typedef struct {
    int32_t op;   /* cg_expr_op */
    int32_t a, b; /* operand node indices (earlier nodes), -1 when unused */
    int32_t i;    /* parameter or input index, or the exponent of POWI */
    double c;     /* the constant of CONST */
} cg_expr_node;

typedef struct cg_expr_program cg_expr_program;

#define CG_EXPR_MAX_NODES 4096
#define CG_EXPR_MAX_INPUTS 4
#define CG_EXPR_MAX_PARAMS 128

/* Generate, compile (NVRTC, loaded at first use) and load the kernels of an
 * expression program on the current device (flags: 0, or CG_EXPR_VALUE_ONLY
 * for a program whose kernels evaluate the objective only; its
 * cg_expr_gradient calls must pass grad = NULL).  *out receives the program
 * (free with cg_expr_free).  CG_ERR_INVALID_ARG for a malformed program
 * (bad operand order or index, a root that does not depend on the
 * elements), CG_ERR_UNSUPPORTED when NVRTC or the driver entry points are
 * unavailable or the elements use more than 127 parameter-only subexpressions
 * (per-thread accumulators), CG_ERR_CUDA when compilation or loading fails.  With
 * CG_ERR_UNSUPPORTED (no NVRTC, driver or device) or CG_ERR_CUDA, *out still
 * receives a program that holds the generated source and the compiler log
 * but cannot run; free it with cg_expr_free. */
#define CG_EXPR_VALUE_ONLY 1   /* flags: objective only (no reverse sweep is generated) */
cg_status cg_expr_compile(const cg_expr_node *nodes, int n_nodes, int n_params, int n_inputs, int flags,
                          cg_expr_program **out);
/* The generated CUDA source and the last compiler log (owned by the program). */
const char *cg_expr_source(const cg_expr_program *prog);
const char *cg_expr_log(const cg_expr_program *prog);
/* Number of per-thread accumulators of the generated tile kernel (1 value +
 * one per parameter-only node the elements use). */
int cg_expr_num_acc(const cg_expr_program *prog);
size_t cg_expr_workspace_size(const cg_expr_program *prog, int64_t n, int64_t n_theta);
/* Objective and gradient at n_theta parameter points.  inputs: host array of
 * n_inputs device pointers, each [n] FP64; theta: device [n_theta][n_params];
 * value: device [n_theta]; grad: device [n_theta][n_params] or NULL (values
 * only).  Asynchronous on stream; capturable in a CUDA graph. */
cg_status cg_expr_gradient(const cg_expr_program *prog, const double *const *inputs, int64_t n,
                           const double *theta, int64_t n_theta, double *value, double *grad, void *ws,
                           size_t ws_bytes, void *stream);
void cg_expr_free(cg_expr_program *prog);

#ifdef __cplusplus
}
#endif

#endif /* CG_H */
