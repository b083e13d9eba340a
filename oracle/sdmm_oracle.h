/*
 * sdmm_oracle.h -- plain FP64 CPU oracle of the SDMM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against what the paper defines ("Path Guiding Using Spatio-Directional
 * Mixture Models", Dodik, Papas, Oztireli, Mueller).  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Everything is FP64 and written as a direct, unblocked loop over samples and
 * components, in the order the paper gives the steps, so that a reader can
 * check it against the equations by eye:
 *
 *   geometry      Sec. 3.1, Eq. (log) and Eq. (exp); App. A (Jacobians)
 *   densities     Sec. 3.1, Eq. (bi-variate), solid-angle change of variables,
 *                 Eq. (solidangle-pdf); "Additional dimensions" paragraph
 *   E-step        Sec. 3.2, Eq. (em-ss-computation), Eq. (tangent-space-mu-update)
 *   M-step        Sec. 3.2 Eq. (em-params-from-ss); Sec. 3.4 "Efficient
 *                 tangent-space covariance update" (first-order transport);
 *                 Sec. 4.3 Eq. (robbins-monroe), Eq. (robbins-monroe-2nd),
 *                 MAP update and prior constants
 *   init          Sec. 4.3 "Initialization"; App. B; App. C
 *   conditioning  Sec. 3.2 (joint fitted, conditioned in closed form), Sec. 3.3
 *   sampling      Sec. 3.1 "Sampling" (discard when |nu| >= pi)
 *
 * Readings where the paper is silent or inconsistent are the ones listed in
 * the repository's design notes; each is restated at the point of use.
 *
 * Array layouts (all row-major, caller-owned):
 *   region r, component k -> index rk = r*K + k
 *   pi[rk], mu_x[rk*3+c], mu_w[rk*3+c] (unit vector), L[rk*15+p]
 *   L and S2 are packed lower triangles, p = i*(i+1)/2 + j for j <= i,
 *   in the 5-D order (x0, x1, x2, nu0, nu1): position first, then direction.
 *
 * Per-region status codes: 0 ok, 1 skipped (fewer than min_samples samples),
 * 2 numeric (a covariance was not positive definite even with the numerical
 * floor; region left unchanged), 3 non-finite statistics, 4 zero total weight,
 * 7 repaired (updated; a covariance needed the numerical floor).
 */
#ifndef SDMM_ORACLE_H
#define SDMM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t K;                /* components per region                          */
    int32_t min_samples;      /* regions with fewer samples are skipped (16)    */
    int32_t eta_mode;         /* 0: Robbins-Monro eta_j, 1: eta = 1 (plain EM)  */
    int32_t estep_density;    /* 0: tangent density p^t (paper), 1: p^Omega     */
    int32_t euclid;           /* 1: (ox, oy) are Euclidean R^2 coordinates      */
    int32_t cov_update;       /* 0: first-order transport, 1: two-pass          */
    int32_t prior_scale_mode; /* 0: beta = 1/n_seen, 1: caller array            */
    int32_t pad_;
    double eta_alpha;         /* 0.5                                            */
    double eta_beta;          /* 0.1                                            */
    double prior_q;           /* q = prior_q / K      (paper: 1)                */
    double prior_a;           /* a = prior_a / K      (paper: 5)                */
    double prior_B_pos;       /* B = a * diag(pos x3, dir x2); paper 1e-4       */
    double prior_B_dir;       /*                                  paper 1e-5    */
} or_config;

typedef struct {
    double  *pi, *mu_x, *mu_w, *L;     /* mixture parameters                 */
    double  *S0, *S2, *Wbar;           /* averaged sufficient statistics     */
    int64_t *n_seen;                   /* distinct samples absorbed (per r)  */
    int32_t *step_j;                   /* Robbins-Monro step index (per r)   */
    int32_t *status;                   /* per-region status                  */
} or_state;

/* ---- geometry (Sec. 3.1, App. A) ------------------------------------- */
double or_sinc(double r);
void   or_basis(const double mu[3], double R[9]);
int    or_log_map(const double mu[3], const double w[3], double nu[2],
                  double *theta, double *s);
void   or_exp_map(const double mu[3], const double nu[2], double w[3]);
void   or_jexp(const double mu[3], const double nu[2], double J[6]);
void   or_jlog(const double mu[3], const double w[3], double J[6]);
int    or_cholesky5(const double S[15], double L[15]);

/* ---- fitting (Sec. 3.2, 3.4, 4.2, 4.3) ------------------------------- */
void or_config_default(or_config *cfg, int K);

int or_estep_region(const or_config *cfg, int K,
                    const double *pi, const double *mu_x, const double *mu_w,
                    const double *L, const double *delta, int64_t M,
                    const float *px, const float *py, const float *pz,
                    const float *ox, const float *oy, const float *oz,
                    const float *w, double *loglik, double *resp,
                    double *s0, double *s1, double *s2, double *W);

int or_fit_regions(const or_config *cfg, int64_t R, const int64_t *offsets,
                   const float *px, const float *py, const float *pz,
                   const float *ox, const float *oy, const float *oz,
                   const float *w, int iters, const double *prior_scale,
                   or_state *st, double *loglik_out);

int or_init_regions(const or_config *cfg, int64_t R, const int64_t *offsets,
                    const float *px, const float *py, const float *pz,
                    const float *w, const double *extent,
                    const double *uniforms, or_state *st);

int or_objective(const or_config *cfg, int64_t R, const int64_t *offsets,
                 const float *px, const float *py, const float *pz,
                 const float *ox, const float *oy, const float *oz,
                 const float *w, const double *prior_scale,
                 const or_state *st, const double *delta, double *F_out,
                 double *g_delta, double *g_L, double *g_logit);

/* ---- queries (Sec. 3.1, 3.2, 3.3) ------------------------------------ */
int or_condition(int K, const double *pi, const double *mu_x,
                 const double *mu_w, const double *L, int64_t Q,
                 const float *qx, const int32_t *region, double *cond_pi,
                 double *cond_m, double *cond_L);

int or_pdf(int K, const double *pi, const double *mu_x, const double *mu_w,
           const double *L, int64_t Q, const float *qx,
           const int32_t *region, const double *dir, double *pdf_out);

int or_sample(int K, const double *pi, const double *mu_x,
              const double *mu_w, const double *L, int64_t Q,
              const float *qx, const int32_t *region, const float *uniforms,
              double *dir_out, double *pdf_out, uint8_t *valid_out,
              int32_t *comp_out, double *margin_out);

/* ---- counter-based RNG (Salmon et al., SC'11) ------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]);
void or_uniforms(uint64_t seed, int64_t Q, float *out3);

#ifdef __cplusplus
}
#endif
#endif
