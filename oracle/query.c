/*
 * query.c -- conditioning, sampling and pdf of a region's mixture at a
 * shading position, FP64 (oracle).  TEST INFRASTRUCTURE ONLY; see
 * sdmm_oracle.h.
 *
 * The joint 5-D mixture is conditioned on the position in closed form
 * (Sec. 3.2: joint fitted, conditioned "using standard closed-form Gaussian
 * conditioning"; Sec. 3.3: only the region's K components).  With the
 * Cholesky factor in (x, nu) order written as L = [[A, 0], [C^T, D]]:
 *   z       = A^{-1} (x - mu^x)
 *   pi'_k  ~ pi_k N_3(x; mu^x, A A^T)
 *   m_k     = C^T z            conditional mean of nu in the mu_k chart
 *   Sigma'_k = D D^T           Schur complement
 * Sampling follows Sec. 3.1 "Sampling": pick k, draw nu ~ N(m_k, D D^T),
 * discard when |nu| >= pi, map with exp_{mu_k}.  The pdf is the solid-angle
 * mixture density Eq. (solidangle-pdf), with p^Omega = p^t / sinc|nu|.
 * (The paper writes p^t sqrt|det G|; sqrt det G equals sinc|nu|, and the
 * change of variables from the chart to the sphere divides by it.)
 */
#include <math.h>
#include <stdlib.h>
#include "sdmm_oracle.h"

#define TWO_PI 6.283185307179586476925286766559
#define PK(i, j) ((i) * ((i) + 1) / 2 + (j))

/* Conditional of component rk at position x: log weight (unnormalised,
   log pi + log N_3), mean m[2], conditional factor D[3] = (d00, d10, d11). */
static double cond_one(const double *pi, const double *mu_x, const double *L,
                       int64_t rk, const double x[3], double m[2], double D[3])
{
    const double *Lk = L + rk * 15;
    double e[3], z[3];
    for (int c = 0; c < 3; ++c) e[c] = x[c] - mu_x[rk * 3 + c];
    /* z = A^{-1} e, forward substitution on the 3x3 block */
    double ldA = 0.0, q = 0.0;
    for (int i = 0; i < 3; ++i) {
        double s = e[i];
        for (int j = 0; j < i; ++j) s -= Lk[PK(i, j)] * z[j];
        z[i] = s / Lk[PK(i, i)];
        q += z[i] * z[i];
        ldA += log(Lk[PK(i, i)]);
    }
    for (int a = 0; a < 2; ++a) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += Lk[PK(3 + a, c)] * z[c];
        m[a] = s;
    }
    D[0] = Lk[PK(3, 3)];
    D[1] = Lk[PK(4, 3)];
    D[2] = Lk[PK(4, 4)];
    if (!(pi[rk] > 0.0)) return -INFINITY;
    return log(pi[rk]) - 0.5 * q - ldA - 1.5 * log(TWO_PI);
}

/* Normalised conditional weights of the K components of one region. */
static void cond_region(int K, const double *pi, const double *mu_x,
                        const double *L, int64_t r, const double x[3],
                        double *cpi, double *cm, double *cD)
{
    double mx = -INFINITY;
    for (int k = 0; k < K; ++k) {
        cpi[k] = cond_one(pi, mu_x, L, r * K + k, x, cm + 2 * k, cD + 3 * k);
        if (cpi[k] > mx) mx = cpi[k];
    }
    double sum = 0.0;
    for (int k = 0; k < K; ++k) {
        cpi[k] = (mx > -INFINITY) ? exp(cpi[k] - mx) : 0.0;
        sum += cpi[k];
    }
    for (int k = 0; k < K; ++k) cpi[k] = sum > 0.0 ? cpi[k] / sum : 0.0;
}

int or_condition(int K, const double *pi, const double *mu_x,
                 const double *mu_w, const double *L, int64_t Q,
                 const float *qx, const int32_t *region, double *cond_pi,
                 double *cond_m, double *cond_L)
{
    (void)mu_w;
    for (int64_t i = 0; i < Q; ++i) {
        double x[3] = { qx[3 * i], qx[3 * i + 1], qx[3 * i + 2] };
        cond_region(K, pi, mu_x, L, region[i], x, cond_pi + i * K,
                    cond_m + i * K * 2, cond_L + i * K * 3);
    }
    return 0;
}

/* Solid-angle pdf of the conditioned mixture at unit direction dir. */
static double pdf_cond(int K, const double *mu_w, int64_t r, const double *cpi,
                       const double *cm, const double *cD, const double dir[3])
{
    double p = 0.0;
    for (int k = 0; k < K; ++k) {
        if (!(cpi[k] > 0.0)) continue;
        double nu[2], th, sn;
        if (or_log_map(mu_w + (r * K + k) * 3, dir, nu, &th, &sn)) continue;
        if (th >= M_PI) continue;
        const double *D = cD + 3 * k;
        double y0 = (nu[0] - cm[2 * k]) / D[0];
        double y1 = (nu[1] - cm[2 * k + 1] - D[1] * y0) / D[2];
        double pt = exp(-0.5 * (y0 * y0 + y1 * y1)) / (TWO_PI * D[0] * D[2]);
        p += cpi[k] * pt / or_sinc(th);
    }
    return p;
}

int or_pdf(int K, const double *pi, const double *mu_x, const double *mu_w,
           const double *L, int64_t Q, const float *qx,
           const int32_t *region, const double *dir, double *pdf_out)
{
    double *cpi = (double *)malloc(sizeof(double) * K);
    double *cm = (double *)malloc(sizeof(double) * 2 * K);
    double *cD = (double *)malloc(sizeof(double) * 3 * K);
    for (int64_t i = 0; i < Q; ++i) {
        double x[3] = { qx[3 * i], qx[3 * i + 1], qx[3 * i + 2] };
        cond_region(K, pi, mu_x, L, region[i], x, cpi, cm, cD);
        pdf_out[i] = pdf_cond(K, mu_w, region[i], cpi, cm, cD, dir + 3 * i);
    }
    free(cpi); free(cm); free(cD);
    return 0;
}

/*
 * One guided sample per query from given uniforms (u0, u1, u2) in [0, 1):
 * component by inverse CDF on u0, nu = m + D z with z by Box-Muller from
 * (1 - u1, u2), valid iff |nu| < pi (Sec. 3.1), dir = exp_{mu_k}(nu), and the
 * pdf at dir (0 when invalid).  comp_out: chosen k; margin_out: distance of
 * u0 * sum(pi') to the nearest CDF boundary (ties are resolved differently
 * by other precisions only within this margin).
 */
int or_sample(int K, const double *pi, const double *mu_x,
              const double *mu_w, const double *L, int64_t Q,
              const float *qx, const int32_t *region, const float *uniforms,
              double *dir_out, double *pdf_out, uint8_t *valid_out,
              int32_t *comp_out, double *margin_out)
{
    double *cpi = (double *)malloc(sizeof(double) * K);
    double *cm = (double *)malloc(sizeof(double) * 2 * K);
    double *cD = (double *)malloc(sizeof(double) * 3 * K);
    for (int64_t i = 0; i < Q; ++i) {
        const int64_t r = region[i];
        double x[3] = { qx[3 * i], qx[3 * i + 1], qx[3 * i + 2] };
        cond_region(K, pi, mu_x, L, r, x, cpi, cm, cD);
        const double u0 = uniforms[3 * i], u1 = uniforms[3 * i + 1], u2 = uniforms[3 * i + 2];
        double tot = 0.0;
        for (int k = 0; k < K; ++k) tot += cpi[k];
        const double t = u0 * tot;
        int kk = -1;
        double cum = 0.0, margin = INFINITY;
        for (int k = 0; k < K; ++k) {
            cum += cpi[k];
            if (fabs(t - cum) < margin) margin = fabs(t - cum);
            if (kk < 0 && t < cum) kk = k;
        }
        if (kk < 0)
            for (int k = K - 1; k >= 0; --k)
                if (cpi[k] > 0.0) { kk = k; break; }
        if (comp_out) comp_out[i] = kk;
        if (margin_out) margin_out[i] = margin;
        if (kk < 0) {
            dir_out[3 * i] = dir_out[3 * i + 1] = dir_out[3 * i + 2] = 0.0;
            pdf_out[i] = 0.0;
            valid_out[i] = 0;
            continue;
        }
        const double rad = sqrt(-2.0 * log(1.0 - u1));
        const double z0 = rad * cos(TWO_PI * u2), z1 = rad * sin(TWO_PI * u2);
        const double *D = cD + 3 * kk;
        double nu[2] = { cm[2 * kk] + D[0] * z0, cm[2 * kk + 1] + D[1] * z0 + D[2] * z1 };
        double dir[3];
        or_exp_map(mu_w + (r * K + kk) * 3, nu, dir);
        for (int c = 0; c < 3; ++c) dir_out[3 * i + c] = dir[c];
        const int valid = sqrt(nu[0] * nu[0] + nu[1] * nu[1]) < M_PI;
        valid_out[i] = (uint8_t)valid;
        pdf_out[i] = valid ? pdf_cond(K, mu_w, r, cpi, cm, cD, dir) : 0.0;
    }
    free(cpi); free(cm); free(cD);
    return 0;
}
