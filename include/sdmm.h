/*
 * sdmm.h -- C ABI of the GB300 (sm_103a) library for spatio-directional
 * Gaussian mixtures, after Dodik, Papas, Oztireli, Mueller, "Path Guiding
 * Using Spatio-Directional Mixture Models".
 *
 * The library fits, per spatial region, a K-component 5-D Gaussian mixture
 * over position x (3-D, Euclidean) and direction w (unit 3-vector, mapped to
 * the 2-D tangent plane at each component's mean by the azimuthal equidistant
 * log map of Sec. 3.1), by weighted, Robbins-Monro averaged MAP-EM
 * (Sec. 3.2, 3.4, 4.2, 4.3).  On the query side it conditions a region's
 * mixture on a shading position, samples a direction and evaluates the
 * solid-angle pdf (Sec. 3.1, 3.3).
 *
 * Conventions shared by every entry point
 *  - Pointers are DEVICE memory allocated and owned by the caller, unless a
 *    parameter says "host".  Configuration structs are host memory and are
 *    read during the call only.  The library keeps no pointer after a call
 *    returns, except inside an sdmm_fit_plan (which binds the workspace and
 *    the state it was created with).
 *  - Calls are asynchronous on `stream`.  Argument errors are detected on the
 *    host before any launch and return SDMM_ERR_INVALID_ARG; nothing is
 *    launched then.  Launch failures return SDMM_ERR_CUDA.  A call never
 *    synchronises the stream, except sdmm_autotune, sdmm_fit_plan_timing and
 *    the kD-tree calls (said there).
 *  - Tracing: with the environment variable SDMM_PROFILE=1 (read once per
 *    process) the fit, objective, query, product and kD-tree entry points
 *    time their launches with CUDA events, wait for them and print
 *    "sdmm: <call> <ms> ms" to stderr; streams being captured are skipped.
 *  - Inputs (const pointers) are never modified.  sdmm_state is in/out.
 *  - The library allocates no device memory: the scratch of every call is
 *    the caller's workspace, whose size sdmm_*_workspace_size reports --
 *    except sdmm_fit_regions_noalloc, which uses a fixed scratch array of
 *    SDMM_NOALLOC_SCRATCH_BYTES compiled into the library.
 *  - Sample streams are structure-of-arrays FP32, sorted by region: region r
 *    owns samples [offsets[r], offsets[r+1]) (offsets: int64, R+1 entries,
 *    device).  Stream pointers need FP32 (4-byte) alignment.
 *  - Mixture arrays are indexed by rk = r*K + k.  The 5-D tangent vector is
 *    ordered (x0, x1, x2, nu0, nu1): position first.  Lower-triangular 5x5
 *    matrices are packed row by row, entry (i, j <= i) at i*(i+1)/2 + j.
 *  - The chart at a unit mean mu rotates mu to +z with R_mu whose rows are
 *    (t, b, mu); (t, b) is the orthonormal basis of Duff et al. (JCGT 2017).
 *    The paper leaves the azimuth of R_mu free; covariances are defined
 *    relative to this choice.
 *  - Errors: the return value; sdmm_last_error() gives a message for the
 *    calling thread.  Per-region outcomes of a fit go to state.status.
 */
#ifndef SDMM_H
#define SDMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *sdmm_stream;

typedef enum {
    SDMM_OK = 0,
    SDMM_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or config      */
    SDMM_ERR_CUDA = 2,          /* a CUDA call failed (message in last_error)  */
    SDMM_ERR_UNSUPPORTED = 4,   /* valid but not implemented (e.g. K > 32)     */
    SDMM_ERR_WORKSPACE = 5      /* workspace smaller than reported size        */
} sdmm_status;

/* Per-region outcome of sdmm_fit_regions / sdmm_init_regions (state.status). */
enum {
    SDMM_REGION_OK = 0,
    SDMM_REGION_SKIPPED = 1,     /* fewer than min_samples samples (Sec. 4.2)   */
    SDMM_REGION_NUMERIC = 2,     /* a covariance was not positive definite even
                                    with the floor below; the failing step left
                                    the region unchanged                        */
    SDMM_REGION_NONFINITE = 3,   /* non-finite weights or statistics            */
    SDMM_REGION_ZERO_WEIGHT = 4, /* all sample weights are zero                 */
    SDMM_REGION_BAD_OFFSETS = 5, /* offsets decrease or exceed N                */
    SDMM_REGION_DEVICE_TIMEOUT = 6, /* a tensor-core wait of the E-step timed out;
                                      no region was updated in that step        */
    SDMM_REGION_REPAIRED = 7     /* updated; a component's MAP covariance was not
                                    positive definite in working precision and
                                    got the smallest tau * B / a (tau = 1e-6,
                                    1e-4, 1e-2, 1) that makes it so; if even
                                    tau = 1 fails the status is NUMERIC        */
};

enum { SDMM_ETA_ROBBINS_MONRO = 0, SDMM_ETA_ONE = 1 };
enum { SDMM_DENSITY_TANGENT = 0, SDMM_DENSITY_SOLID_ANGLE = 1 };
enum { SDMM_PRIOR_SCALE_SEEN = 0, SDMM_PRIOR_SCALE_ARRAY = 1 };
enum { SDMM_PREC_FP32 = 0, SDMM_PREC_TC_3XBF16 = 1, SDMM_PREC_TC_TF32 = 2,
       SDMM_PREC_TC_3XTF32 = 3, SDMM_PREC_TC_6XBF16 = 4 };
enum { SDMM_COV_FIRST_ORDER = 0, SDMM_COV_TWO_PASS = 1 };
/* Directional coordinates of the fit: the tangent chart of each component
   (the paper, Sec. 3.1), or, as an ablation without any change of
   variables, the first two world coordinates of the direction,
   nu = (w_x - mu_x, w_y - mu_y), with the new mean mu + (m_x, m_y, 0) and no
   chart transport. */
enum { SDMM_DIR_TANGENT = 0, SDMM_DIR_EUCLIDEAN = 1 };

#define SDMM_MAX_K 32
/* Floats per component in the derived FP32 tables (see sdmm_state). */
#define SDMM_ETAB_FLOATS 36
#define SDMM_QTAB_FLOATS 36

typedef struct sdmm_config {
    int32_t K;                 /* components per region, 1..32                */
    int32_t min_samples;       /* smaller regions are skipped; paper: 16      */
    int32_t eta_mode;          /* SDMM_ETA_*: Robbins-Monro step sizes
                                  eta_j = (eta_beta j + 1)^-eta_alpha
                                  (Sec. 4.3 Eq. robbins-monroe), or eta = 1
                                  (plain EM on a fixed batch)                 */
    int32_t estep_density;     /* SDMM_DENSITY_*: responsibilities from the
                                  tangent density p^t (paper, Eq. em-ss-
                                  computation) or the solid-angle density     */
    int32_t prior_scale_mode;  /* SDMM_PRIOR_SCALE_*: beta = 1/n_seen, or the
                                  caller's per-region array                   */
    int32_t precision;         /* SDMM_PREC_*: E-step arithmetic.  FP32: SIMT
                                  kernel.  TC_*: contraction form on the
                                  tensor cores (K = 16 or 32, either
                                  density): per-sample features times a
                                  per-region coefficient matrix in split
                                  3xBF16 (two BF16 pieces, three products),
                                  TF32, split 3xTF32, or 6xBF16 (three BF16
                                  pieces, the six products of order <= 2),
                                  statistics as a second product in split
                                  3xBF16, FP32 accumulation in TMEM          */
    int32_t chunk;             /* samples per work unit of the fit kernels;
                                  0 = library heuristic; else a multiple of
                                  256 in [256, 65536]                        */
    int32_t ctas_per_sm;       /* resident CTAs per SM of the persistent fit
                                  kernels; 0 = library default, else 1..4.
                                  The E-step of the fit and of the objective
                                  for K >= 3 runs one grid of every resident
                                  CTA (five 4-warp CTAs per SM) and ignores
                                  it; it applies to the adjoint, the second
                                  pass of the two-pass update and K <= 2     */
    int32_t cov_update;        /* SDMM_COV_*: the covariance of the new mean's
                                  chart from the first-order chart change of
                                  the averaged statistics (Sec. 3.4, default),
                                  or the accurate update (Sec. 3.2 Eq.
                                  tangent-space-sigma-update): a second pass
                                  over the batch measures it in the new chart
                                  with the same responsibilities.  The
                                  accurate update is defined for plain EM
                                  (eta_mode = SDMM_ETA_ONE; the batch is the
                                  statistic) and runs on the FP32 SIMT path   */
    int32_t dir_coords;        /* SDMM_DIR_*: tangent charts (default) or the
                                  Euclidean ablation (fit and objective only;
                                  queries, product sampling and the two-pass
                                  update reject it, and of the tensor-core
                                  forms it runs on 6xBF16 and 3xTF32:
                                  SDMM_ERR_UNSUPPORTED)                       */
    double eta_alpha;          /* 0.5 (Sec. 4.3)                              */
    double eta_beta;           /* 0.1 (Sec. 4.3)                              */
    double prior_q;            /* Dirichlet prior q = prior_q / K; paper 1    */
    double prior_a;            /* Wishart prior a = prior_a / K; paper 5      */
    double prior_B_pos;        /* B = a diag(pos, pos, pos, dir, dir);        */
    double prior_B_dir;        /*   paper pos 1e-4, dir 1e-5 (Sec. 4.3)       */
} sdmm_config;

/*
 * Mixture state of R regions x K components.  All device pointers, caller-
 * owned, sized as noted (rk = r*K + k).
 *   pi[RK]          weights                                   (FP64)
 *   mu_x[RK*3]      spatial means                             (FP64)
 *   mu_w[RK*3]      directional means, unit vectors           (FP64)
 *   L[RK*15]        Cholesky factor of the 5-D covariance in the mu_w chart,
 *                   packed lower, (x, nu) order               (FP64)
 *   S0[RK], S2[RK*15]  averaged statistics (Sec. 4.3): weight and centred
 *                   second moment in the current chart; the averaged first
 *                   moment is zero by construction            (FP64)
 *   Wbar[R]         averaged mean sample weight               (FP64)
 *   n_seen[R]       samples absorbed so far (beta = 1/n_seen) (int64)
 *   step_j[R]       Robbins-Monro step index                  (int32)
 *   status[R]       SDMM_REGION_* of the last fit/init        (int32)
 *   etab[RK*SDMM_ETAB_FLOATS], qtab[RK*SDMM_QTAB_FLOATS]
 *                   derived FP32 records read by the E-step and the query
 *                   kernels; written by every successful M-step and by
 *                   sdmm_prepare.  Layout is private to the library; 16-byte
 *                   aligned.
 * The FP64 arrays are the checkpoint: saving them and calling sdmm_prepare
 * after a reload restores the tables.
 */
typedef struct sdmm_state {
    double *pi, *mu_x, *mu_w, *L;
    double *S0, *S2, *Wbar;
    int64_t *n_seen;
    int32_t *step_j;
    int32_t *status;
    float *etab, *qtab;
} sdmm_state;

/* A batch of weighted samples (path vertices; Sec. 4.2): x = (px, py, pz),
   w = (ox, oy, oz) unit, weight w >= 0 (incident-radiance estimate). */
typedef struct sdmm_samples {
    const float *px, *py, *pz, *ox, *oy, *oz, *w;  /* [N] each, device     */
    const int64_t *offsets;                         /* [R+1], device       */
    int64_t R;                                      /* regions             */
    int64_t N;                                      /* offsets[R] <= N     */
} sdmm_samples;

/* Uniform grid of regions over an axis-aligned box: region of x is
   ix + dims[0]*(iy + dims[1]*iz), i = clamp(floor((x - lo)*scale), 0, dims-1),
   scale = dims / (hi - lo) evaluated in FP32. */
typedef struct sdmm_grid {
    float lo[3], hi[3];
    int32_t dims[3];
} sdmm_grid;

/* Fills `cfg` with the paper's constants for K components (Sec. 4.2, 4.3). */
void sdmm_config_default(sdmm_config *cfg, int32_t K);

/* Thread-local message for the last error of this thread ("" if none). */
const char *sdmm_last_error(void);

/* Library version string. */
const char *sdmm_version(void);

/*
 * Bytes of workspace that sdmm_fit_regions / sdmm_objective /
 * sdmm_objective_backward / sdmm_fit_plan_create need for R regions and N
 * samples with this configuration (chunk size included).  Host call.
 */
sdmm_status sdmm_fit_workspace_size(const sdmm_config *cfg, int64_t R,
                                    int64_t N, size_t *bytes);

/*
 * Mixture initialisation (Sec. 4.3 "Initialization", App. B, App. C) for
 * regions with at least min_samples samples: n_pos = K/8 spatial seeds (1 if
 * 8 does not divide K) by weighted k-means++ on position with weights
 * clamp(w, 0.1, 3) and Euclidean distance; n_dir = K/n_pos directions (cube
 * corners when 8, else a Fibonacci spiral); Sigma^x = (2 d / n_pos)^2 I3 /
 * chi2_3^{-1}(0.9), Sigma^nu = (2 pi / n_dir) I2, pi = 1/K, statistics reset.
 * Surface normals are not available, so the spatial part is isotropic.
 *   extent[R]     device FP64, longest side d of each region's cell
 *   uniforms[R*n_pos]  device FP64 in [0, 1): the k-means++ draws
 * Regions below min_samples get status SKIPPED and are otherwise untouched.
 * The seed choice is computed in FP64 in sequential order.  Updates etab/qtab.
 */
sdmm_status sdmm_init_regions(const sdmm_config *cfg, const sdmm_samples *s,
                              const double *extent, const double *uniforms,
                              sdmm_state *st, sdmm_stream stream);

/*
 * `iters` EM steps of every region on this batch (Sec. 4.2 "Mini-batch EM
 * fitting"; one launch of each fit kernel per step):
 *   E-step  responsibilities from pi_k p_k(d_ki), d_ki = (x_i - mu_k^x,
 *           log_{mu_k}(w_i)), per-sample log-sum-exp in FP32
 *           (Sec. 3.2 Eq. em-ss-computation)
 *   stats   weighted sums of [1, d, d d^T] per component, FP32 per work unit,
 *           reduced in FP64 in a fixed order (deterministic)
 *   average S^ = (1 - eta_j) S^ + eta_j S/W (Sec. 4.3 Eq. robbins-monroe),
 *           eta_0 = 1
 *   M-step  FP64: mean offset m = S^1/S^0, mu^x += m^x, mu_w = exp_{mu_w}(m^nu)
 *           (Eq. tangent-space-mu-update); centred second moment moved to the
 *           new chart by J = J_log(mu_new) J_exp_{mu_old}(m^nu) (Sec. 3.4,
 *           App. A); MAP pi = (beta q + S^0)/(K beta q + sum S^0), Sigma =
 *           (beta B + S^2)/(beta a + S^0) (Sec. 4.3); 5x5 Cholesky.
 * beta = prior_scale[r] (device FP64 [R], prior_scale_mode ARRAY) or
 * 1/n_seen with n_seen counting this batch once.  loglik_out (nullable,
 * device FP32 [N]) receives the per-sample log-likelihood of the last E-step
 * (entries of skipped regions are left untouched).  Regions whose status is
 * not OK after the first step are not updated by later steps of the call.
 * workspace: device, 256-byte aligned, >= sdmm_fit_workspace_size bytes.
 */
sdmm_status sdmm_fit_regions(const sdmm_config *cfg, const sdmm_samples *s,
                             int32_t iters, const double *prior_scale,
                             sdmm_state *st, float *loglik_out,
                             void *workspace, size_t ws_bytes,
                             sdmm_stream stream);

/* Rebuild the FP32 tables etab/qtab of all R regions from the FP64
   parameters (after the caller wrote or reloaded pi, mu_x, mu_w, L).
   logits (nullable, device FP64 [RK]): first sets pi = softmax(logits) per
   region.  delta (nullable, device FP64 [RK*5]): the E-step records then
   evaluate each component at the mean offset delta inside its own chart,
   density N(d - delta; 0, Sigma), as sdmm_objective does for its gradient
   (the query records and the FP64 parameters are not offset).  A later
   M-step rewrites the records without offset. */
sdmm_status sdmm_prepare(const sdmm_config *cfg, int64_t R, sdmm_state *st,
                         const double *logits, const double *delta,
                         sdmm_stream stream);

/*
 * Conditioning on position (Sec. 3.2: closed-form Gaussian conditioning of
 * the joint; Sec. 3.3: the K components of the query's region).  With
 * L = [[A, 0], [C^T, D]] (position block A), per query i and component k:
 *   cond_pi[i*K+k]      pi'_k ~ pi_k N_3(x; mu^x, A A^T), normalised
 *   cond_m[(i*K+k)*2]   conditional mean of nu in the mu_k chart, C^T A^-1 (x - mu^x)
 *   cond_L[(i*K+k)*3]   conditional Cholesky factor D = (d00, d10, d11)
 * qx: device FP32 [Q*3]; region: device int32 [Q] or NULL, then `grid`
 * (host) maps positions to regions.  Region ids must be < R; the tables of
 * state `st` must be prepared for R regions.
 */
sdmm_status sdmm_condition(const sdmm_config *cfg, const sdmm_state *st,
                           int64_t R, int64_t Q, const float *qx,
                           const int32_t *region, const sdmm_grid *grid,
                           float *cond_pi, float *cond_m, float *cond_L,
                           sdmm_stream stream);

/*
 * One guided direction per query (Sec. 3.1 "Sampling"): condition, pick k by
 * inverse CDF on u0, nu = m_k + D_k z with z from Box-Muller on (1 - u1, u2),
 * discard when |nu| >= pi (valid = 0, pdf = 0), dir = exp_{mu_k}(nu), and
 * the solid-angle pdf of the conditioned mixture at dir (Eq. solidangle-pdf,
 * p^Omega = p^t / sinc|nu|).  Uniforms: `uniforms` (device FP32 [Q*3]) if
 * not NULL, else Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 * counter = (i, 0, 0): u = (word >> 8) * 2^-24 for words 0..2.
 * Outputs (device): dir_out FP32 [Q*3], pdf_out FP32 [Q], valid_out u8 [Q].
 */
sdmm_status sdmm_sample(const sdmm_config *cfg, const sdmm_state *st,
                        int64_t R, int64_t Q, const float *qx,
                        const int32_t *region, const sdmm_grid *grid,
                        uint64_t seed, const float *uniforms, float *dir_out,
                        float *pdf_out, uint8_t *valid_out,
                        sdmm_stream stream);

/* Solid-angle pdf of the conditioned mixture at given unit directions
   dir (device FP32 [Q*3]) (Eq. solidangle-pdf); pdf_out device FP32 [Q]. */
sdmm_status sdmm_pdf(const sdmm_config *cfg, const sdmm_state *st, int64_t R,
                     int64_t Q, const float *qx, const int32_t *region,
                     const sdmm_grid *grid, const float *dir, float *pdf_out,
                     sdmm_stream stream);

/*
 * sdmm_sample and sdmm_pdf for queries in any order, binned by region inside
 * the library (Sec. 3.3: every query reads its region's K components; queries
 * of one region then share those reads).  A counting sort of the queries by
 * region runs in the caller's workspace (device memory of at least
 * sdmm_query_workspace_size(R, Q) bytes, 256-byte aligned, clobbered), then
 * the queries are processed region by region; every output goes to the
 * query's own index, and the result of a query depends only on its inputs and
 * its index (the Philox counter), so it equals that of sdmm_sample / sdmm_pdf
 * up to the order-independent rounding of the pdf sum.  Arguments, uniforms,
 * outputs and errors as for sdmm_sample / sdmm_pdf; in addition Q must be
 * below 2^31 (SDMM_ERR_INVALID_ARG) and a workspace that is NULL, misaligned
 * or too small is SDMM_ERR_WORKSPACE.  With K > 16 the queries are processed
 * in the given order and the workspace is not used.
 */
sdmm_status sdmm_query_workspace_size(int64_t R, int64_t Q, size_t *bytes);
sdmm_status sdmm_sample_binned(const sdmm_config *cfg, const sdmm_state *st,
                               int64_t R, int64_t Q, const float *qx,
                               const int32_t *region, const sdmm_grid *grid,
                               uint64_t seed, const float *uniforms,
                               float *dir_out, float *pdf_out,
                               uint8_t *valid_out, void *workspace,
                               size_t ws_bytes, sdmm_stream stream);
sdmm_status sdmm_pdf_binned(const sdmm_config *cfg, const sdmm_state *st,
                            int64_t R, int64_t Q, const float *qx,
                            const int32_t *region, const sdmm_grid *grid,
                            const float *dir, float *pdf_out, void *workspace,
                            size_t ws_bytes, sdmm_stream stream);

/*
 * Weighted MAP objective per region (the function that the MAP-EM of
 * Sec. 4.3 ascends; Dirichlet and inverse-Wishart priors after Gauvain-Lee):
 *   F_r = (1/W) sum_i w_i l_i + sum_k [beta q log pi_k - (beta a/2) log|Sigma_k|
 *         - (beta/2) tr(B Sigma_k^-1)],   l_i = log sum_k pi_k p_k(d_ki).
 * F_out: device FP64 [R].  beta as in sdmm_fit_regions (1/n_seen without
 * counting a new batch; 0 when n_seen = 0).  workspace as for the fit.
 */
sdmm_status sdmm_objective(const sdmm_config *cfg, const sdmm_samples *s,
                           const double *prior_scale, const sdmm_state *st,
                           double *F_out, void *workspace, size_t ws_bytes,
                           sdmm_stream stream);

/*
 * Adjoint of sdmm_objective: given dF (device FP64 [R]), writes
 * dF_r * dF_r/d(theta) for every component (device FP32):
 *   g_delta[RK*5]  w.r.t. an offset delta of the mean inside the component's
 *                  own chart (density N(d - delta; 0, Sigma)), at the offset
 *                  the E-step records carry (0 unless set by sdmm_prepare)
 *   g_L[RK*15]     w.r.t. the packed Cholesky factor L
 *   g_logit[RK]    w.r.t. logits a with pi = softmax(a) per region
 * The paper has no gradients; this is the derivative of the objective above.
 */
sdmm_status sdmm_objective_backward(const sdmm_config *cfg,
                                    const sdmm_samples *s,
                                    const double *prior_scale,
                                    const sdmm_state *st, const double *dF,
                                    float *g_delta, float *g_L,
                                    float *g_logit, void *workspace,
                                    size_t ws_bytes, sdmm_stream stream);

/*
 * Fit plan: the per-step launch sequence of sdmm_fit_regions for a fixed
 * configuration, region count, maximum sample count, state and workspace,
 * captured once into a CUDA graph and replayed per batch.  The batch (sample
 * pointers, offsets, N) is passed per run and written to a device descriptor
 * inside the workspace by a small kernel before the replay, so fresh batches
 * need no re-capture.  Create captures on `stream` (which must not be
 * capturing already).  Host handle; destroy frees only host-side objects.
 */
typedef struct sdmm_fit_plan sdmm_fit_plan;

sdmm_status sdmm_fit_plan_create(const sdmm_config *cfg, int64_t R,
                                 int64_t N_max, int32_t iters,
                                 sdmm_state *st, void *workspace,
                                 size_t ws_bytes, sdmm_stream stream,
                                 sdmm_fit_plan **plan_out);
/* Runs the plan on batch `s` (s->R must equal the plan's R, s->N <= N_max).
   prior_scale and loglik_out as in sdmm_fit_regions; like the sample
   pointers they may differ from run to run.  Runs on one plan must not
   overlap on the GPU (they share the plan's workspace). */
sdmm_status sdmm_fit_plan_run(sdmm_fit_plan *plan, const sdmm_samples *s,
                              const double *prior_scale, float *loglik_out,
                              sdmm_stream stream);
/* Batches from host memory (Sec. 4.2: the renderer produces each round's
   samples on the host).  sdmm_fit_plan_run_host copies the seven sample
   arrays and the offsets of `host_batch` (host pointers; pinned memory for
   asynchronous copies) into one of two slots of `staging` (device,
   caller-owned, 256-byte aligned, sdmm_fit_plan_staging_size bytes) on a copy
   stream owned by the plan, then replays the plan on `stream` once the copy
   is done.  Consecutive runs alternate the slots, so the copy of the next
   batch overlaps the replay of the previous one; a slot is rewritten only
   after the replay that read it.  The host arrays must stay unchanged until
   `stream` has passed the run.  Device pointers in `host_batch` are
   rejected (SDMM_ERR_INVALID_ARG); a small or misaligned staging buffer gives
   SDMM_ERR_WORKSPACE. */
sdmm_status sdmm_fit_plan_staging_size(const sdmm_fit_plan *plan, size_t *bytes_out);
sdmm_status sdmm_fit_plan_run_host(sdmm_fit_plan *plan, const sdmm_samples *host_batch,
                                   void *staging, size_t staging_bytes,
                                   const double *prior_scale, float *loglik_out,
                                   sdmm_stream stream);
/* Enable per-run event timing of the E-step kernel of each step inside the
   graph, for up to `capacity` runs before sdmm_fit_plan_timing is read. */
sdmm_status sdmm_fit_plan_enable_timing(sdmm_fit_plan *plan, int32_t capacity);
/* Synchronises the plan's events and writes, host-side, the E-step kernel
   durations (ms) of the runs since the last read: ms_out[*n_out]. */
sdmm_status sdmm_fit_plan_timing(sdmm_fit_plan *plan, float *ms_out,
                                 int32_t max, int32_t *n_out);
sdmm_status sdmm_fit_plan_destroy(sdmm_fit_plan *plan);

/*
 * Autotuner: times the E-step kernel on this batch for candidate chunk sizes
 * and CTAs per SM (without touching the state's parameters; the statistics
 * go to the workspace) and returns the fastest pair.  Where the E-step
 * ignores ctas_per_sm (K >= 3) only the chunk is tuned and *ctas_per_sm_out
 * is 0 (the default).  Synchronises `stream`.
 * The workspace must be sized for the largest candidate: use
 * sdmm_fit_workspace_size with chunk = 256.
 */
sdmm_status sdmm_autotune(const sdmm_config *cfg, const sdmm_samples *s,
                          const sdmm_state *st, void *workspace,
                          size_t ws_bytes, sdmm_stream stream,
                          int32_t *chunk_out, int32_t *ctas_per_sm_out,
                          float *best_ms_out);

/*
 * Self-test of the tensor-core contraction path: D = A B^T for one tile with
 * A (128 x Kd) and B (N x Kd) given in FP32 (device, row-major), rounded to
 * the operand format `kind` (0: BF16, tcgen05.mma kind::f16; 1: TF32,
 * kind::tf32), staged in shared memory in the same K-major layout and
 * multiplied with the same descriptors, MMA issue, commit and TMEM read-out
 * as the contraction-form E-step; D (device FP32, 128 x N) accumulates in
 * FP32.  N: multiple of 16 in [16, 256]; Kd: multiple of 16 (BF16) or 8
 * (TF32), at most 64.  `variant` bits: 1 swaps the two descriptor offsets of
 * K-major operands (diagnostics), 2 / 4 stage A / B MN-major (BF16 only),
 * 8 swaps the offsets of MN-major operands (diagnostics), 16 makes A 64 x Kd
 * (M = 64; D then holds all 128 TMEM lanes, showing where the 64 rows sit).
 * Variants 0, 4 and 6 are the layouts the contraction-form E-step uses.
 * status (device int32): set to 1 if the MMA did not complete within 2 s.
 * (The paper has no counterpart: this checks the hardware path.)
 */
/*
 * Input validation (the fit itself does not check samples): counts[0] =
 * samples whose direction is not unit length within unit_tol (|w|^2 - 1
 * beyond 2 unit_tol), counts[1] = weights negative or not finite, counts[2] =
 * positions not finite; counts is device int64[3], overwritten.  offsets and
 * R are not used.  Asynchronous.
 */
sdmm_status sdmm_validate_samples(const sdmm_samples *s, float unit_tol, int64_t *counts,
                                  sdmm_stream stream);

/*
 * Failure detection without a fault: the bounded mbarrier wait that every
 * tensor-core wait of the E-step uses, on a barrier that completes only when
 * `arrive` is non-zero.  With nobody arriving the wait gives up after
 * limit_ns (1 .. 2e9), writes *status = 1 (device int32) and the elapsed time
 * (*elapsed_ns, device int64) and the kernel returns normally, leaving the
 * context usable; with an arrival *status = 0.  (The E-step reports the same
 * event as region status SDMM_REGION_DEVICE_TIMEOUT.)  Asynchronous.
 */
sdmm_status sdmm_wait_selftest(int64_t limit_ns, int32_t arrive, int32_t *status,
                               int64_t *elapsed_ns, sdmm_stream stream);

sdmm_status sdmm_tc_selftest(int32_t kind, int32_t N, int32_t Kd,
                             const float *A, const float *B, float *D,
                             int32_t variant, int32_t *status,
                             sdmm_stream stream);

/*
 * sdmm_fit_regions_noalloc -- the fit of sdmm_fit_regions for callers that
 * may not allocate device memory.  (The paper has no counterpart: this entry
 * point only concerns where the library's scratch memory comes from.)
 *
 * Who needs it: code that must not call cudaMalloc or any allocating routine
 * -- e.g. a renderer plugin whose host application owns and budgets all
 * device memory, code running inside an allocator or driver callback where
 * allocating would re-enter the allocator, or a real-time loop that must
 * never block on an allocation.  Such callers can still pass the inputs and
 * outputs they already own.
 *
 * Instead of a caller workspace, the call uses a fixed scratch array of
 * SDMM_NOALLOC_SCRATCH_BYTES compiled into this library; every GPU on which
 * the library is loaded holds that array until the process exits.  The
 * function itself calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *  - Limit: problems whose scratch (sdmm_fit_workspace_size for the same
 *    cfg, R and N) exceeds SDMM_NOALLOC_SCRATCH_BYTES are rejected with
 *    SDMM_ERR_WORKSPACE and a message giving both sizes; nothing is launched.
 *    With K = 16 this allows roughly 12,000 work units, e.g. 4,096 regions with
 *    up to about 30M samples, or one region with up to 3M samples.
 *  - Set-up: the first call on each device looks up the device address of the
 *    scratch array (cudaGetSymbolAddress, with that device current) and
 *    caches it; make that first call before any stream capture.
 *  - Sharing: all calls on a device share the one array, which keeps the
 *    last call's contents.  Each call writes every scratch byte it reads
 *    before reading it, so nothing needs clearing between calls, but calls
 *    whose work overlaps on the GPU (other streams, other host threads)
 *    race on the scratch and produce wrong results: serialise them.
 * Arguments, results and per-region statuses are those of sdmm_fit_regions
 * (every precision and covariance update); with the same cfg the results are
 * bit-identical to it, since both cut the regions into the same work units.
 */
#define SDMM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
sdmm_status sdmm_fit_regions_noalloc(const sdmm_config *cfg,
                                     const sdmm_samples *s, int32_t iters,
                                     const double *prior_scale,
                                     sdmm_state *st, float *loglik_out,
                                     sdmm_stream stream);

/*
 * ---- Product sampling with a BSDF mixture (Sec. 3.5 "Product Sampling from
 * Mixed-Orientation Gaussians", Eq. product-distribution; Sec. 4.1 "Pruning
 * before product sampling").
 *
 * Each query carries J BSDF lobes, already conditioned and rotated by the
 * caller into the frame of the radiance mixtures: weight w (>= 0), unit mean
 * direction mu (3 floats) and the packed lower Cholesky factor (l00, l10, l11)
 * of the lobe's covariance in its own chart (the Duff basis of mu, as for the
 * radiance components).  Only the two lobes of largest weight are used (lower
 * index on ties).  Every (radiance component k, lobe j) pair is formed in the
 * chart of mu_k with the lobe's covariance moved by J = J_log_{mu_k}(mu_j)
 * J_exp_{mu_j}(0); the product of the two Gaussians there is one Gaussian of
 * weight pi'_k w_j N(m_k; log_{mu_k}(mu_j), S1 + J S2 J^T).  A lobe at the
 * antipode of mu_k makes no pair.
 */
typedef struct sdmm_bsdf_lobes {
    const float *w;      /* [Q*J] lobe weights                              */
    const float *mu;     /* [Q*J*3] unit mean directions                    */
    const float *L;      /* [Q*J*3] (l00, l10, l11) in the lobe's chart     */
    int32_t J;           /* lobes per query, 1..8                           */
} sdmm_bsdf_lobes;

/* One direction per query from the product mixture: the pair by inverse CDF
   on u0 (pairs ordered by component, then lobe index), a Gaussian draw in its
   chart (Box-Muller on 1 - u1, u2), |nu| >= pi discarded (valid = 0, pdf 0),
   omega = exp_{mu_k}(nu); pdf_out = the product mixture's density on the
   sphere at omega.  Uniforms as in sdmm_sample. */
sdmm_status sdmm_product_sample(const sdmm_config *cfg, const sdmm_state *st, int64_t R,
                                int64_t Q, const float *qx, const int32_t *region,
                                const sdmm_grid *grid, const sdmm_bsdf_lobes *bsdf,
                                uint64_t seed, const float *uniforms, float *dir_out,
                                float *pdf_out, uint8_t *valid_out, sdmm_stream stream);

/* Density on the sphere of the product mixture at given unit directions
   (dir[3Q]): the sum over pairs of weight N(log_{mu_k}(omega)) / sinc. */
sdmm_status sdmm_product_pdf(const sdmm_config *cfg, const sdmm_state *st, int64_t R,
                             int64_t Q, const float *qx, const int32_t *region,
                             const sdmm_grid *grid, const sdmm_bsdf_lobes *bsdf,
                             const float *dir, float *pdf_out, sdmm_stream stream);

/*
 * ---- The spatial kD-tree of the regions (Sec. 4.2 "Refinement of the
 * spatial kD-tree", Sec. 4.3 "Initialization").
 *
 * Positions are normalised to [0,1]^3 (the scene's bounding box, Sec. 4.3).
 * The tree is a device array of nodes; node 0 is the root.  A leaf node has
 * axis -1 and the index of its region in `leaf`; an internal node sends
 * x[axis] < split to `left` and the rest to left + 1.  Leaves are numbered in
 * tree order (left before right), so once samples are sorted by leaf the
 * samples of leaf r form the r-th contiguous segment (the region offsets of
 * sdmm_fit_regions).  The counts are host fields updated by the calls;
 * capacities are the lengths of the arrays.
 */
typedef struct sdmm_kdtree {
    int32_t *axis;       /* [cap_nodes] split axis 0..2, or -1 for a leaf   */
    double *split;       /* [cap_nodes] split position                      */
    int32_t *left;       /* [cap_nodes] first child (the second: left + 1)  */
    int32_t *leaf;       /* [cap_nodes] region index of a leaf node         */
    int32_t n_nodes;     /* nodes in use (host field)                       */
    int32_t n_leaves;    /* leaves = regions (host field)                   */
    int32_t cap_nodes;
    int32_t cap_leaves;
} sdmm_kdtree;

/* Sample streams written by the tree calls (device, caller-owned): N floats
   each and offsets[cap_leaves + 1]; R and N are set by the call. */
typedef struct sdmm_sample_buffers {
    float *px, *py, *pz, *ox, *oy, *oz, *w;
    int64_t *offsets;
    int64_t R;
    int64_t N;
} sdmm_sample_buffers;

/* The pre-subdivision of Sec. 4.3: every axis split at the centre of its cell,
   x then y then z, `levels` times (3: the paper's 8 x 8 x 8 cells).  Needs
   cap_nodes >= 2^(3 levels + 1) - 1 and cap_leaves >= 8^levels; levels 0..7.
   Leaf r is the cell whose Morton code (bits x y z, most significant first)
   is r.  Synchronous on `stream`. */
sdmm_status sdmm_kdtree_grid(sdmm_kdtree *t, int32_t levels, sdmm_stream stream);

/* Region of Q points (device SoA) by descent from the root; writes leaf[Q]
   (int32).  Asynchronous. */
sdmm_status sdmm_kdtree_lookup(const sdmm_kdtree *t, int64_t Q, const float *px,
                               const float *py, const float *pz, int32_t *leaf,
                               sdmm_stream stream);

/* Workspace bytes of sdmm_kdtree_bin / sdmm_kdtree_refine for N samples with
   this tree's capacities (N < 2^31). */
sdmm_status sdmm_kdtree_workspace_size(const sdmm_kdtree *t, int64_t N, size_t *bytes);

/* Binning (Sec. 4.2: each leaf collects the vertices located within it): the
   N samples of `in` (any order; in->offsets and in->R are ignored) sorted by
   leaf into `out`, stably (original order within a leaf), with
   out->offsets[n_leaves + 1]: every sample's leaf by descent, a stable radix
   sort by leaf, one gather of the seven streams.  Synchronous on `stream`. */
sdmm_status sdmm_kdtree_bin(const sdmm_kdtree *t, const sdmm_samples *in,
                            sdmm_sample_buffers *out, void *workspace,
                            size_t ws_bytes, sdmm_stream stream);

/* Refinement (Sec. 4.2): every leaf holding more than c samples is split along
   the axis of largest positional variance at the mean position along it,
   recursively, until no leaf holds more than c or a split would leave one
   side empty (the paper uses c = 16000).  Mean and variance come from exact
   fixed-point sums (x clamped to [0,1], in units of 2^-32), so the planes do
   not depend on summation order.  `in` holds the samples sorted by the
   current leaves (in->R = t->n_leaves, in->offsets); `out` receives them
   sorted by the new leaves (stable) with out->offsets; leaf_parent[cap_leaves]
   (int64) receives for every new leaf the leaf of the input it lies in (copy
   its mixture with sdmm_gather_regions, as the paper copies the parent's).
   The tree is updated in place: split leaves become internal nodes, new
   nodes are appended, leaves are renumbered in tree order.  At most 64 split
   rounds (tree levels) per call; SDMM_ERR_WORKSPACE if the capacities would
   be exceeded (the tree is then left as before the failing round).
   Synchronous on `stream`. */
sdmm_status sdmm_kdtree_refine(sdmm_kdtree *t, int64_t c, const sdmm_samples *in,
                               sdmm_sample_buffers *out, int64_t *leaf_parent,
                               void *workspace, size_t ws_bytes, sdmm_stream stream);

/* out region r <- in region src[r] for r < R_out: parameters, averaged
   statistics, Wbar, n_seen, step_j, status and the derived tables (K
   components each).  `in` and `out` must not overlap.  Asynchronous. */
sdmm_status sdmm_gather_regions(int32_t K, int64_t R_out, const int64_t *src,
                                const sdmm_state *in, sdmm_state *out,
                                sdmm_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SDMM_H */
