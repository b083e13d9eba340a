/*
 * em.c -- weighted, averaged MAP-EM of 5-D spatio-directional mixtures,
 * FP64 (oracle).  TEST INFRASTRUCTURE ONLY; see sdmm_oracle.h.
 *
 * Per region and per call: one batch of M weighted samples (x, w, weight),
 * `iters` EM steps.  Each step:
 *   E   responsibilities S_ki = pi_k p_k^t(d_ki) / sum_l pi_l p_l^t(d_li)
 *       with d_ki = (x_i - mu_k^x, log_{mu_k}(w_i))      Sec. 3.2 Eq. (em-ss-computation)
 *   SS  s0 = sum w S, s1 = sum w S d, s2 = sum w S d d^T, all / sum w
 *   EMA S^ = (1 - eta_j) S^_{j-1} + eta_j S             Sec. 4.3 Eq. (robbins-monroe)
 *   M   mean through the exp map                         Sec. 3.2 Eq. (tangent-space-mu-update)
 *       centred second moment moved to the new chart by the first-order
 *       Jacobian                                         Sec. 3.4, Sec. 4.3 Eq. (robbins-monroe-2nd)
 *       MAP weights / covariances                        Sec. 4.3 (MAP EM)
 *
 * Readings (the paper is silent or inconsistent):
 *  - eta weights the NEW batch (Eq. robbins-monroe); the index j starts at 0 on
 *    a region's first step, so eta_0 = 1; the same rule is used for the second
 *    moment (Eq. robbins-monroe-2nd swaps the roles, read as a typo).
 *  - The stored second moment is centred at the new mean and expressed in the
 *    new chart; the stored first moment is therefore zero.  The chart change
 *    uses T = blockdiag(I3, J), J = D(log_{mu_new} o exp_{mu_old}) at m^nu,
 *    i.e. J_log(mu_new) * J_exp(m^nu) (App. A), mapping old chart to new.
 *  - beta_j = 1 / n_seen, n_seen = distinct samples absorbed by the region.
 *  - The averaged normalisation factor is tracked as an EMA of W/M (mean
 *    weight); it does not enter the M-step since pi, mu and Sigma are ratios.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "sdmm_oracle.h"

#define TWO_PI 6.283185307179586476925286766559
#define PK(i, j) ((i) * ((i) + 1) / 2 + (j))
/* inverse CDF of chi-square with 3 degrees of freedom at 0.9 (App. B) */
#define CHI2_3_Q90 6.2513886311703222

void or_config_default(or_config *cfg, int K)
{
    memset(cfg, 0, sizeof(*cfg));
    cfg->K = K;
    cfg->min_samples = 16;           /* Sec. 4.2: leaves with M >= 16 */
    cfg->eta_mode = 0;
    cfg->estep_density = 0;          /* Eq. (em-ss-computation) uses p^t */
    cfg->euclid = 0;
    cfg->cov_update = 0;
    cfg->prior_scale_mode = 0;
    cfg->eta_alpha = 0.5;            /* Sec. 4.3 */
    cfg->eta_beta = 0.1;
    cfg->prior_q = 1.0;              /* Sec. 4.3: q = 1/K */
    cfg->prior_a = 5.0;              /*            a = 5/K */
    cfg->prior_B_pos = 1e-4;         /* B = a diag(0.1, 0.1, 1, 1, 1) 1e-4 */
    cfg->prior_B_dir = 1e-5;         /*   in the paper's (nu, x) order      */
}

/* 5-D tangent vector d = (x - mu^x, log_mu(w)); returns 1 on the cut locus. */
static int tangent5(const or_config *cfg, const double *mux, const double *muw,
                    const double x[3], const double wd[3], double d[5],
                    double *logjac)
{
    for (int c = 0; c < 3; ++c) d[c] = x[c] - mux[c];
    *logjac = 0.0;
    if (cfg->euclid) {
        d[3] = wd[0] - muw[0];
        d[4] = wd[1] - muw[1];
        return 0;
    }
    double th, sn;
    if (or_log_map(muw, wd, d + 3, &th, &sn)) return 1;
    /* solid-angle density divides p^t by sinc|nu| = sn/th (Sec. 3.1) */
    if (cfg->estep_density == 1 && sn > 0.0) *logjac = log(th / sn);
    return 0;
}

/* y = L^{-1} d by forward substitution. */
static void lower_solve5(const double *L, const double d[5], double y[5])
{
    for (int i = 0; i < 5; ++i) {
        double e = d[i];
        for (int j = 0; j < i; ++j) e -= L[PK(i, j)] * y[j];
        y[i] = e / L[PK(i, i)];
    }
}

/* z = L^{-T} y by back substitution. */
static void upper_solve5(const double *L, const double y[5], double z[5])
{
    for (int i = 4; i >= 0; --i) {
        double e = y[i];
        for (int j = i + 1; j < 5; ++j) e -= L[PK(j, i)] * z[j];
        z[i] = e / L[PK(i, i)];
    }
}

/* log N_5(d; 0, L L^T) */
static double lognormal5(const double *L, const double d[5], double y[5])
{
    lower_solve5(L, d, y);
    double q = 0.0, ld = 0.0;
    for (int i = 0; i < 5; ++i) {
        q += y[i] * y[i];
        ld += log(L[PK(i, i)]);
    }
    return -0.5 * q - ld - 2.5 * log(TWO_PI);
}

/*
 * E-step for one region (Sec. 3.2, Eq. em-ss-computation): per-sample
 * log-likelihood l_i = log sum_k pi_k p_k(d_ki), responsibilities and the
 * raw (un-normalised) weighted statistics s0[K], s1[5K], s2[15K] (packed),
 * and W = sum w.  `delta` (nullable, 5K) offsets each component's mean inside
 * its own chart (used by the objective's gradient check).  `resp` (nullable,
 * M*K) receives the responsibilities.
 */
int or_estep_region(const or_config *cfg, int K, const double *pi,
                    const double *mu_x, const double *mu_w, const double *L,
                    const double *delta, int64_t M, const float *px,
                    const float *py, const float *pz, const float *ox,
                    const float *oy, const float *oz, const float *w,
                    double *loglik, double *resp, double *s0, double *s1,
                    double *s2, double *W)
{
    double *lk = (double *)malloc(sizeof(double) * K);
    double *dk = (double *)malloc(sizeof(double) * 5 * K);
    if (!lk || !dk) { free(lk); free(dk); return 1; }
    for (int k = 0; k < K; ++k) {
        s0[k] = 0.0;
        for (int a = 0; a < 5; ++a) s1[k * 5 + a] = 0.0;
        for (int p = 0; p < 15; ++p) s2[k * 15 + p] = 0.0;
    }
    *W = 0.0;
    for (int64_t i = 0; i < M; ++i) {
        double x[3] = { px[i], py[i], pz[i] };
        double wd[3] = { ox[i], oy[i], oz[i] };
        double wt = w[i];
        *W += wt;
        double mx = -INFINITY;
        for (int k = 0; k < K; ++k) {
            double *d = dk + 5 * k, y[5], lj;
            if (tangent5(cfg, mu_x + 3 * k, mu_w + 3 * k, x, wd, d, &lj) ||
                !(pi[k] > 0.0)) {
                lk[k] = -INFINITY;
                continue;
            }
            if (delta)
                for (int a = 0; a < 5; ++a) d[a] -= delta[5 * k + a];
            lk[k] = log(pi[k]) + lognormal5(L + 15 * k, d, y) + lj;
            if (lk[k] > mx) mx = lk[k];
        }
        double li = -INFINITY;
        if (mx > -INFINITY) {
            double sum = 0.0;
            for (int k = 0; k < K; ++k) sum += exp(lk[k] - mx);
            li = mx + log(sum);
        }
        if (loglik) loglik[i] = li;
        for (int k = 0; k < K; ++k) {
            double r = (li > -INFINITY) ? exp(lk[k] - li) : 0.0;
            if (resp) resp[i * K + k] = r;
            if (r == 0.0) continue;
            double wr = wt * r;
            const double *d = dk + 5 * k;
            s0[k] += wr;
            for (int a = 0; a < 5; ++a) {
                s1[k * 5 + a] += wr * d[a];
                for (int b = 0; b <= a; ++b) s2[k * 15 + PK(a, b)] += wr * d[a] * d[b];
            }
        }
    }
    free(lk);
    free(dk);
    return 0;
}

/* C = A B for small dense row-major matrices. */
static void matmul(int n, int m, int p, const double *A, const double *B, double *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < p; ++j) {
            double e = 0.0;
            for (int l = 0; l < m; ++l) e += A[i * m + l] * B[l * p + j];
            C[i * p + j] = e;
        }
}

static void unpack5(const double *P, double S[25])
{
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) S[i * 5 + j] = S[j * 5 + i] = P[PK(i, j)];
}

/*
 * Chart change of a centred second moment (Sec. 3.4, Sec. 4.3): the
 * direction block is mapped by J = J_log_{mu_new}(mu_new) J_exp_{mu_old}(m),
 * the position block is left as is: C' = T C T^T, T = blockdiag(I3, J).
 */
static void transport_cov(const or_config *cfg, const double *mu_old,
                          const double *mu_new, const double m_nu[2],
                          const double Cpk[15], double out[15])
{
    double T[25] = { 0 };
    for (int c = 0; c < 3; ++c) T[c * 5 + c] = 1.0;
    if (cfg->euclid) {
        T[3 * 5 + 3] = T[4 * 5 + 4] = 1.0;
    } else {
        double Je[6], Jl[6], J[4];
        or_jexp(mu_old, m_nu, Je);
        or_jlog(mu_new, mu_new, Jl);
        matmul(2, 3, 2, Jl, Je, J);
        T[3 * 5 + 3] = J[0]; T[3 * 5 + 4] = J[1];
        T[4 * 5 + 3] = J[2]; T[4 * 5 + 4] = J[3];
    }
    double C[25], TC[25], TCT[25], Tt[25];
    unpack5(Cpk, C);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Tt[i * 5 + j] = T[j * 5 + i];
    matmul(5, 5, 5, T, C, TC);
    matmul(5, 5, 5, TC, Tt, TCT);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) out[PK(i, j)] = 0.5 * (TCT[i * 5 + j] + TCT[j * 5 + i]);
}

/* One EM step of one region; statistics are the raw sums from the E-step. */
static int mstep_region(const or_config *cfg, int K, int64_t r, int64_t M,
                        const double *s0, const double *s1, const double *s2,
                        double W, const double *s2_two_pass, double beta,
                        or_state *st)
{
    const int64_t base = r * K;
    double eta = 1.0;
    if (cfg->eta_mode == 0)
        eta = pow(cfg->eta_beta * (double)st->step_j[r] + 1.0, -cfg->eta_alpha);
    const double q = cfg->prior_q / K, a = cfg->prior_a / K;
    const double Bd[5] = { a * cfg->prior_B_pos, a * cfg->prior_B_pos, a * cfg->prior_B_pos,
                           a * cfg->prior_B_dir, a * cfg->prior_B_dir };

    double *nS0 = (double *)malloc(sizeof(double) * K);
    double *nS2 = (double *)malloc(sizeof(double) * 15 * K);
    double *nmx = (double *)malloc(sizeof(double) * 3 * K);
    double *nmw = (double *)malloc(sizeof(double) * 3 * K);
    double *nL = (double *)malloc(sizeof(double) * 15 * K);
    double *npi = (double *)malloc(sizeof(double) * K);
    int bad = 0, repaired = 0;
    double sumS0 = 0.0;
    for (int k = 0; k < K && !bad; ++k) {
        const int64_t rk = base + k;
        /* batch statistics normalised by the total weight, Eq. (em-ss-computation) */
        double S0 = s0[k] / W, S1[5], S2[15];
        for (int c = 0; c < 5; ++c) S1[c] = s1[k * 5 + c] / W;
        for (int p = 0; p < 15; ++p) S2[p] = s2[k * 15 + p] / W;
        /* Robbins-Monro averaging, Eq. (robbins-monroe); stored S1 is zero */
        double hS0 = (1.0 - eta) * st->S0[rk] + eta * S0;
        double hS1[5], hS2[15];
        for (int c = 0; c < 5; ++c) hS1[c] = eta * S1[c];
        for (int p = 0; p < 15; ++p) hS2[p] = (1.0 - eta) * st->S2[rk * 15 + p] + eta * S2[p];
        int nonfinite = !isfinite(hS0);
        for (int p = 0; p < 15; ++p) if (!isfinite(hS2[p])) nonfinite = 1;
        for (int c = 0; c < 5; ++c) if (!isfinite(hS1[c])) nonfinite = 1;
        if (nonfinite) { bad = 3; break; }
        /* mean offset in the current chart and new mean, Eq. (tangent-space-mu-update) */
        double m[5];
        for (int c = 0; c < 5; ++c) m[c] = hS0 > 0.0 ? hS1[c] / hS0 : 0.0;
        for (int c = 0; c < 3; ++c) nmx[k * 3 + c] = st->mu_x[rk * 3 + c] + m[c];
        if (cfg->euclid) {
            nmw[k * 3 + 0] = st->mu_w[rk * 3 + 0] + m[3];
            nmw[k * 3 + 1] = st->mu_w[rk * 3 + 1] + m[4];
            nmw[k * 3 + 2] = st->mu_w[rk * 3 + 2];
        } else {
            or_exp_map(st->mu_w + rk * 3, m + 3, nmw + k * 3);
        }
        if (s2_two_pass) {
            /* accurate update, Eq. (tangent-space-sigma-update): statistics
               recomputed in the new chart, already centred at the new mean */
            for (int p = 0; p < 15; ++p) nS2[k * 15 + p] = s2_two_pass[k * 15 + p] / W;
        } else {
            /* centred second moment in the old chart, then first-order chart
               change (Sec. 3.4 "Efficient tangent-space covariance update") */
            double C[15];
            for (int i = 0; i < 5; ++i)
                for (int j = 0; j <= i; ++j) C[PK(i, j)] = hS2[PK(i, j)] - hS0 * m[i] * m[j];
            transport_cov(cfg, st->mu_w + rk * 3, nmw + k * 3, m + 3, C, nS2 + k * 15);
        }
        nS0[k] = hS0;
        sumS0 += hS0;
        /* MAP covariance, Sec. 4.3 */
        double Sig[15];
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j <= i; ++j)
                Sig[PK(i, j)] = ((i == j ? beta * Bd[i] : 0.0) + nS2[k * 15 + PK(i, j)]) /
                                (beta * a + hS0);
        if (or_cholesky5(Sig, nL + k * 15)) {
            /* Numerical floor (reading; the paper's prior is meant to stop
               collapse but vanishes as beta -> 0): add the smallest of
               tau * B / a, tau = 1e-6, 1e-4, 1e-2, 1, that makes the
               covariance positive definite; the region is flagged. */
            int fixed = 0;
            for (double tau = 1e-6; tau <= 1.0 && !fixed; tau *= 100.0) {
                double S2f[15];
                for (int p = 0; p < 15; ++p) S2f[p] = Sig[p];
                for (int c = 0; c < 5; ++c) S2f[PK(c, c)] += tau * Bd[c] / a;
                fixed = !or_cholesky5(S2f, nL + k * 15);
            }
            if (fixed) repaired = 1;
            else bad = 2;
        }
    }
    if (!bad) {
        /* MAP weights, Sec. 4.3 */
        for (int k = 0; k < K; ++k)
            npi[k] = (beta * q + nS0[k]) / (K * beta * q + sumS0);
        for (int k = 0; k < K; ++k) {
            const int64_t rk = base + k;
            st->pi[rk] = npi[k];
            for (int c = 0; c < 3; ++c) {
                st->mu_x[rk * 3 + c] = nmx[k * 3 + c];
                st->mu_w[rk * 3 + c] = nmw[k * 3 + c];
            }
            for (int p = 0; p < 15; ++p) {
                st->L[rk * 15 + p] = nL[k * 15 + p];
                st->S2[rk * 15 + p] = nS2[k * 15 + p];
            }
            st->S0[rk] = nS0[k];
        }
        st->Wbar[r] = (1.0 - eta) * st->Wbar[r] + eta * (W / (double)M);
        st->step_j[r] += 1;
    }
    free(nS0); free(nS2); free(nmx); free(nmw); free(nL); free(npi);
    return bad ? bad : (repaired ? 7 : 0);
}

/*
 * Fit all regions on one batch: `iters` EM steps per region (Sec. 4.2
 * "Mini-batch EM fitting").  Regions are independent.  Samples of region r
 * are [offsets[r], offsets[r+1]).  loglik_out (nullable, N) receives the
 * per-sample log-likelihood of the last E-step.
 */
int or_fit_regions(const or_config *cfg, int64_t R, const int64_t *offsets,
                   const float *px, const float *py, const float *pz,
                   const float *ox, const float *oy, const float *oz,
                   const float *w, int iters, const double *prior_scale,
                   or_state *st, double *loglik_out)
{
    const int K = cfg->K;
    double *s0 = (double *)malloc(sizeof(double) * K);
    double *s1 = (double *)malloc(sizeof(double) * 5 * K);
    double *s2 = (double *)malloc(sizeof(double) * 15 * K);
    double *s2b = (double *)malloc(sizeof(double) * 15 * K);
    if (!s0 || !s1 || !s2 || !s2b) return 1;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t o = offsets[r], M = offsets[r + 1] - offsets[r];
        if (M < cfg->min_samples) { st->status[r] = 1; continue; }
        double Wsum = 0.0;
        for (int64_t i = 0; i < M; ++i) Wsum += w[o + i];
        if (!isfinite(Wsum)) { st->status[r] = 3; continue; }
        if (!(Wsum > 0.0)) { st->status[r] = 4; continue; }
        /* the batch counts once towards n_seen, committed with the first
           successful step; a failing step leaves the region as it was */
        const int64_t seen = st->n_seen[r] + M;
        double beta = (cfg->prior_scale_mode == 1 && prior_scale)
                          ? prior_scale[r] : 1.0 / (double)seen;
        int status = 0;
        double *resp = NULL;
        if (cfg->cov_update == 1) resp = (double *)malloc(sizeof(double) * M * K);
        int worst = 0;
        for (int it = 0; it < iters && (status == 0 || status == 7); ++it) {
            double W;
            const int64_t rk = r * K;
            or_estep_region(cfg, K, st->pi + rk, st->mu_x + rk * 3, st->mu_w + rk * 3,
                            st->L + rk * 15, NULL, M, px + o, py + o, pz + o, ox + o,
                            oy + o, oz + o, w + o,
                            (loglik_out && it == iters - 1) ? loglik_out + o : NULL,
                            resp, s0, s1, s2, &W);
            const double *two = NULL;
            if (cfg->cov_update == 1) {
                /* second pass: the batch re-mapped into each new mean's chart,
                   with the responsibilities of this E-step */
                for (int k = 0; k < K * 15; ++k) s2b[k] = 0.0;
                for (int k = 0; k < K; ++k) {
                    double m[5], nmx[3], nmw[3];
                    for (int c = 0; c < 5; ++c) m[c] = s0[k] > 0.0 ? s1[k * 5 + c] / s0[k] : 0.0;
                    for (int c = 0; c < 3; ++c) nmx[c] = st->mu_x[(rk + k) * 3 + c] + m[c];
                    if (cfg->euclid) {
                        nmw[0] = st->mu_w[(rk + k) * 3 + 0] + m[3];
                        nmw[1] = st->mu_w[(rk + k) * 3 + 1] + m[4];
                        nmw[2] = st->mu_w[(rk + k) * 3 + 2];
                    } else {
                        or_exp_map(st->mu_w + (rk + k) * 3, m + 3, nmw);
                    }
                    for (int64_t i = 0; i < M; ++i) {
                        double x[3] = { px[o + i], py[o + i], pz[o + i] };
                        double wd[3] = { ox[o + i], oy[o + i], oz[o + i] };
                        double d[5], lj;
                        if (tangent5(cfg, nmx, nmw, x, wd, d, &lj)) continue;
                        double wr = w[o + i] * resp[i * K + k];
                        for (int a = 0; a < 5; ++a)
                            for (int b = 0; b <= a; ++b) s2b[k * 15 + PK(a, b)] += wr * d[a] * d[b];
                    }
                }
                two = s2b;
            }
            status = mstep_region(cfg, K, r, M, s0, s1, s2, W, two, beta, st);
            if (status == 0 || status == 7) st->n_seen[r] = seen;
            if (status == 7) worst = 7;
        }
        free(resp);
        st->status[r] = (status == 0 && worst) ? worst : status;
    }
    free(s0); free(s1); free(s2); free(s2b);
    return 0;
}

/* Index chosen by inverse CDF on non-negative weights p (sequential sum). */
static int64_t pick_index(const double *p, int64_t M, double u)
{
    double tot = 0.0;
    for (int64_t i = 0; i < M; ++i) tot += p[i];
    if (!(tot > 0.0)) return -1;
    double t = u * tot, cum = 0.0;
    int64_t last = -1;
    for (int64_t i = 0; i < M; ++i) {
        cum += p[i];
        if (p[i] > 0.0) last = i;
        if (t < cum) return i;
    }
    return last;
}

/*
 * Mixture initialisation (Sec. 4.3 "Initialization", App. B, App. C), with
 * the readings for data without surface normals:
 *  - n_pos = K/8 spatial seeds (2 for K = 16) picked by weighted k-means++ on
 *    position: the first with probability proportional to clamp(w, 0.1, 3),
 *    each next one proportional to clamp(w, 0.1, 3) times the Euclidean
 *    distance to the closest seed so far (App. C); uniforms are inputs,
 *    n_pos per region.  K not divisible by 8: one spatial seed.
 *  - directions: the 8 cube corners (+-1, +-1, +-1)/sqrt(3) when there are
 *    8 per seed, otherwise a Fibonacci spiral of n_dir points.
 *  - Sigma^x = r_st^2 I3 / chi2_3^{-1}(0.9), r_st = 2 d / n_pos (App. B; no
 *    normal, so isotropic), d = longest side of the region (extent[r]).
 *  - Sigma^nu = (2 pi / n_dir) I2 (App. B), pi = 1/K.
 * Averaged statistics, n_seen and step_j are reset.
 */
int or_init_regions(const or_config *cfg, int64_t R, const int64_t *offsets,
                    const float *px, const float *py, const float *pz,
                    const float *w, const double *extent,
                    const double *uniforms, or_state *st)
{
    const int K = cfg->K;
    const int n_pos = (K % 8 == 0) ? K / 8 : 1;
    const int n_dir = K / n_pos;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t o = offsets[r], M = offsets[r + 1] - offsets[r];
        st->n_seen[r] = 0;
        st->step_j[r] = 0;
        st->Wbar[r] = 0.0;
        for (int64_t rk = r * K; rk < (r + 1) * K; ++rk) {
            st->S0[rk] = 0.0;
            for (int p = 0; p < 15; ++p) st->S2[rk * 15 + p] = 0.0;
        }
        if (M < cfg->min_samples) { st->status[r] = 1; continue; }
        double *p = (double *)malloc(sizeof(double) * M);
        double *dmin = (double *)malloc(sizeof(double) * M);
        int64_t seed[64];
        for (int64_t i = 0; i < M; ++i) {
            double c = w[o + i];
            c = c < 0.1 ? 0.1 : (c > 3.0 ? 3.0 : c);
            p[i] = c;
            dmin[i] = INFINITY;
        }
        seed[0] = pick_index(p, M, uniforms[r * n_pos + 0]);
        for (int j = 1; j < n_pos; ++j) {
            const int64_t s = seed[j - 1];
            double *q = (double *)malloc(sizeof(double) * M);
            for (int64_t i = 0; i < M; ++i) {
                double dx = (double)px[o + i] - (double)px[o + s];
                double dy = (double)py[o + i] - (double)py[o + s];
                double dz = (double)pz[o + i] - (double)pz[o + s];
                double dd = sqrt(dx * dx + dy * dy + dz * dz);
                if (dd < dmin[i]) dmin[i] = dd;
                q[i] = p[i] * dmin[i];
            }
            int64_t nxt = pick_index(q, M, uniforms[r * n_pos + j]);
            seed[j] = nxt < 0 ? seed[0] : nxt;
            free(q);
        }
        const double rst = 2.0 * extent[r] / n_pos;
        const double sx = rst / sqrt(CHI2_3_Q90);
        const double sw = sqrt(TWO_PI / n_dir);
        for (int j = 0; j < n_pos; ++j) {
            for (int t = 0; t < n_dir; ++t) {
                const int64_t rk = r * K + j * n_dir + t;
                double dvec[3];
                if (n_dir == 8) {
                    const double h = 1.0 / sqrt(3.0);
                    dvec[0] = (t & 1) ? -h : h;
                    dvec[1] = (t & 2) ? -h : h;
                    dvec[2] = (t & 4) ? -h : h;
                } else {
                    const double ga = M_PI * (3.0 - sqrt(5.0));
                    double z = 1.0 - (2.0 * t + 1.0) / n_dir;
                    double rad = sqrt(1.0 - z * z);
                    dvec[0] = rad * cos(ga * t);
                    dvec[1] = rad * sin(ga * t);
                    dvec[2] = z;
                }
                st->pi[rk] = 1.0 / K;
                st->mu_x[rk * 3 + 0] = px[o + seed[j]];
                st->mu_x[rk * 3 + 1] = py[o + seed[j]];
                st->mu_x[rk * 3 + 2] = pz[o + seed[j]];
                for (int c = 0; c < 3; ++c) st->mu_w[rk * 3 + c] = dvec[c];
                for (int q = 0; q < 15; ++q) st->L[rk * 15 + q] = 0.0;
                for (int c = 0; c < 3; ++c) st->L[rk * 15 + PK(c, c)] = sx;
                for (int c = 3; c < 5; ++c) st->L[rk * 15 + PK(c, c)] = sw;
            }
        }
        st->status[r] = 0;
        free(p);
        free(dmin);
    }
    return 0;
}

/*
 * Weighted MAP objective per region (derived from Sec. 4.3, MAP EM after
 * Gauvain and Lee): the weighted mean log-likelihood plus the log of the
 * Dirichlet and inverse-Wishart priors whose stationary point is the MAP
 * update of Sec. 4.3,
 *   F = (1/W) sum_i w_i l_i
 *     + sum_k [ beta q log pi_k - (beta a / 2) log|Sigma_k| - (beta/2) tr(B Sigma_k^{-1}) ].
 * Gradients (nullable outputs) with respect to the in-chart mean offset
 * delta_k (5), the packed Cholesky factor L_k (15) and weight logits a_k
 * with pi = softmax(a):
 *   dF/d delta_k = sum_i wt_i r_ik z_ik,  y = L^{-1} d, z = L^{-T} y
 *   dF/dL_k      = tril(sum_i wt_i r_ik (z y^T - diag(1/L_jj)))
 *                  - beta a diag(1/L_jj) + beta tril(Sigma^{-1} B L^{-T})
 *   dF/da_k      = sum_i wt_i (r_ik - pi_k) + beta q (1 - K pi_k)
 * with wt_i = w_i / W.  beta as in the fit (1/n_seen, or caller array).
 */
int or_objective(const or_config *cfg, int64_t R, const int64_t *offsets,
                 const float *px, const float *py, const float *pz,
                 const float *ox, const float *oy, const float *oz,
                 const float *w, const double *prior_scale,
                 const or_state *st, const double *delta, double *F_out,
                 double *g_delta, double *g_L, double *g_logit)
{
    const int K = cfg->K;
    const double q = cfg->prior_q / K, a = cfg->prior_a / K;
    const double Bd[5] = { a * cfg->prior_B_pos, a * cfg->prior_B_pos, a * cfg->prior_B_pos,
                           a * cfg->prior_B_dir, a * cfg->prior_B_dir };
    double *lk = (double *)malloc(sizeof(double) * K);
    double *yk = (double *)malloc(sizeof(double) * 5 * K);
    double *dk = (double *)malloc(sizeof(double) * 5 * K);
    for (int64_t r = 0; r < R; ++r) {
        const int64_t o = offsets[r], M = offsets[r + 1] - offsets[r];
        const int64_t rk0 = r * K;
        double beta;
        if (cfg->prior_scale_mode == 1 && prior_scale) beta = prior_scale[r];
        else beta = st->n_seen[r] > 0 ? 1.0 / (double)st->n_seen[r] : 0.0;
        double W = 0.0;
        for (int64_t i = 0; i < M; ++i) W += w[o + i];
        if (g_delta) for (int64_t t = 0; t < 5 * K; ++t) g_delta[rk0 * 5 + t] = 0.0;
        if (g_L) for (int64_t t = 0; t < 15 * K; ++t) g_L[rk0 * 15 + t] = 0.0;
        if (g_logit) for (int k = 0; k < K; ++k) g_logit[rk0 + k] = 0.0;
        double F = 0.0;
        if (W > 0.0) {
            for (int64_t i = 0; i < M; ++i) {
                double x[3] = { px[o + i], py[o + i], pz[o + i] };
                double wd[3] = { ox[o + i], oy[o + i], oz[o + i] };
                double mx = -INFINITY;
                for (int k = 0; k < K; ++k) {
                    const int64_t rk = rk0 + k;
                    double lj, *d = dk + 5 * k;
                    if (tangent5(cfg, st->mu_x + rk * 3, st->mu_w + rk * 3, x, wd, d, &lj) ||
                        !(st->pi[rk] > 0.0)) {
                        lk[k] = -INFINITY;
                        continue;
                    }
                    if (delta) for (int c = 0; c < 5; ++c) d[c] -= delta[rk * 5 + c];
                    lk[k] = log(st->pi[rk]) + lognormal5(st->L + rk * 15, d, yk + 5 * k) + lj;
                    if (lk[k] > mx) mx = lk[k];
                }
                if (!(mx > -INFINITY)) continue;
                double sum = 0.0;
                for (int k = 0; k < K; ++k) sum += exp(lk[k] - mx);
                const double li = mx + log(sum);
                const double wt = w[o + i] / W;
                F += wt * li;
                for (int k = 0; k < K; ++k) {
                    const int64_t rk = rk0 + k;
                    const double rr = exp(lk[k] - li);
                    if (g_logit) g_logit[rk] += wt * (rr - st->pi[rk]);
                    if (rr == 0.0) continue;
                    const double *L = st->L + rk * 15;
                    double z[5];
                    upper_solve5(L, yk + 5 * k, z);
                    if (g_delta)
                        for (int c = 0; c < 5; ++c) g_delta[rk * 5 + c] += wt * rr * z[c];
                    if (g_L)
                        for (int ii = 0; ii < 5; ++ii)
                            for (int jj = 0; jj <= ii; ++jj) {
                                double gv = z[ii] * yk[5 * k + jj];
                                if (ii == jj) gv -= 1.0 / L[PK(ii, ii)];
                                g_L[rk * 15 + PK(ii, jj)] += wt * rr * gv;
                            }
                }
            }
        }
        /* prior terms */
        for (int k = 0; k < K; ++k) {
            const int64_t rk = rk0 + k;
            const double *L = st->L + rk * 15;
            /* Linv columns: Linv e_j, so Sigma^{-1} = Linv^T Linv */
            double Li[25] = { 0 }, Sinv[25], e[5], col[5];
            for (int j = 0; j < 5; ++j) {
                for (int c = 0; c < 5; ++c) e[c] = (c == j) ? 1.0 : 0.0;
                lower_solve5(L, e, col);
                for (int c = 0; c < 5; ++c) Li[c * 5 + j] = col[c];
            }
            for (int i = 0; i < 5; ++i)
                for (int j = 0; j < 5; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < 5; ++c) s += Li[c * 5 + i] * Li[c * 5 + j];
                    Sinv[i * 5 + j] = s;
                }
            double logdet = 0.0, trBS = 0.0;
            for (int j = 0; j < 5; ++j) {
                logdet += 2.0 * log(L[PK(j, j)]);
                trBS += Bd[j] * Sinv[j * 5 + j];
            }
            F += beta * q * log(st->pi[rk]) - 0.5 * beta * a * logdet - 0.5 * beta * trBS;
            if (g_logit) g_logit[rk] += beta * q * (1.0 - K * st->pi[rk]);
            if (g_L) {
                /* beta tril(Sigma^{-1} B L^{-T}); (L^{-T})_{jc} = Li[c][j] */
                for (int ii = 0; ii < 5; ++ii)
                    for (int jj = 0; jj <= ii; ++jj) {
                        double s = 0.0;
                        for (int c = 0; c < 5; ++c) s += Sinv[ii * 5 + c] * Bd[c] * Li[jj * 5 + c];
                        double gv = beta * s;
                        if (ii == jj) gv -= beta * a / L[PK(ii, ii)];
                        g_L[rk * 15 + PK(ii, jj)] += gv;
                    }
            }
        }
        F_out[r] = F;
    }
    free(lk); free(yk); free(dk);
    return 0;
}
