/*
 * geom.c -- tangent-space geometry of the sphere, FP64 (oracle).
 * TEST INFRASTRUCTURE ONLY; see sdmm_oracle.h.
 *
 * Sec. 3.1 defines the chart at a unit mean mu by the azimuthal equidistant
 * projection: rotate by R_mu (which takes mu to +z), then scale the xy part
 * so that its length equals the geodesic angle to mu (Eq. log); the exp map
 * walks back (Eq. exp).  sinc is the unnormalised sin(r)/r.
 */
#include <math.h>
#include "sdmm_oracle.h"

/* sinc(r) = sin(r)/r, unnormalised (Sec. 3.1); Taylor series near 0. */
double or_sinc(double r)
{
    if (fabs(r) < 1e-4) {
        double r2 = r * r;
        return 1.0 - r2 / 6.0 + r2 * r2 / 120.0;
    }
    return sin(r) / r;
}

/*
 * R_mu: a rotation taking mu to +z (Sec. 3.1).  The paper leaves its azimuth
 * free.  Reading: rows (t, b, mu), where (t, b) is the branchless
 * orthonormal basis of Duff et al., "Building an Orthonormal Basis,
 * Revisited" (JCGT 6(1), 2017), restated from that paper's formulas.
 */
void or_basis(const double mu[3], double R[9])
{
    double sgn = copysign(1.0, mu[2]);
    double a = -1.0 / (sgn + mu[2]);
    double b = mu[0] * mu[1] * a;
    R[0] = 1.0 + sgn * mu[0] * mu[0] * a;
    R[1] = sgn * b;
    R[2] = -sgn * mu[0];
    R[3] = b;
    R[4] = sgn + mu[1] * mu[1] * a;
    R[5] = -mu[1];
    R[6] = mu[0];
    R[7] = mu[1];
    R[8] = mu[2];
}

/*
 * log_mu(w), Eq. (log): w' = R_mu w, nu = w'_xy / sinc(angle(w', z)).
 * The angle is taken as atan2(|w'_xy|, w'_z), which equals acos(w'_z) for a
 * unit vector and keeps full accuracy near 0 and pi.  Returns 1 when w is
 * the antipode of mu (the cut locus, where the chart is undefined), else 0.
 * Optionally reports theta = |nu| and s = |w'_xy|.
 */
int or_log_map(const double mu[3], const double w[3], double nu[2],
               double *theta, double *s)
{
    double R[9];
    or_basis(mu, R);
    double u = R[0] * w[0] + R[1] * w[1] + R[2] * w[2];
    double v = R[3] * w[0] + R[4] * w[1] + R[5] * w[2];
    double c = R[6] * w[0] + R[7] * w[1] + R[8] * w[2];
    double sn = sqrt(u * u + v * v);
    double th = atan2(sn, c);
    if (theta) *theta = th;
    if (s) *s = sn;
    if (sn == 0.0) {
        nu[0] = 0.0;
        nu[1] = 0.0;
        return c > 0.0 ? 0 : 1;
    }
    /* 1/sinc(th) applied to the unit-length w'_xy: |nu| = th exactly */
    double g = th / sn;
    nu[0] = g * u;
    nu[1] = g * v;
    return 0;
}

/* exp_mu(nu), Eq. (exp): w = R_mu^T (nu sinc|nu|, cos|nu|). */
void or_exp_map(const double mu[3], const double nu[2], double w[3])
{
    double R[9];
    or_basis(mu, R);
    double r = sqrt(nu[0] * nu[0] + nu[1] * nu[1]);
    double sc = or_sinc(r);
    double p[3] = { nu[0] * sc, nu[1] * sc, cos(r) };
    for (int c = 0; c < 3; ++c)
        w[c] = R[0 * 3 + c] * p[0] + R[1 * 3 + c] * p[1] + R[2 * 3 + c] * p[2];
}

/*
 * Jacobian of exp_mu at nu (App. A), a 3x2 matrix, row-major J[3][2].
 * App. A prints the (1,2) entry with an extra sinc term and the (2,2) entry
 * without the square; differentiating Eq. (exp) gives instead
 *   R_mu^T [[s + nx^2 c, nx ny c], [nx ny c, s + ny^2 c], [-nx s, -ny s]]
 * with s = sinc r and c = (cos r - s)/r^2 (limit -1/3 + r^2/30 at r -> 0).
 */
void or_jexp(const double mu[3], const double nu[2], double J[6])
{
    double R[9];
    or_basis(mu, R);
    double r2 = nu[0] * nu[0] + nu[1] * nu[1];
    double r = sqrt(r2);
    double s = or_sinc(r);
    double c;
    if (r < 1e-2)
        c = -1.0 / 3.0 + r2 / 30.0 - r2 * r2 / 840.0;
    else
        c = (cos(r) - s) / r2;
    double Jp[6] = {
        s + nu[0] * nu[0] * c, nu[0] * nu[1] * c,
        nu[0] * nu[1] * c,     s + nu[1] * nu[1] * c,
        -nu[0] * s,            -nu[1] * s,
    };
    for (int row = 0; row < 3; ++row)
        for (int col = 0; col < 2; ++col)
            J[row * 2 + col] = R[0 * 3 + row] * Jp[0 * 2 + col] +
                               R[1 * 3 + row] * Jp[1 * 2 + col] +
                               R[2 * 3 + row] * Jp[2 * 2 + col];
}

/*
 * Jacobian of log_mu at w (App. A), a 2x3 matrix, row-major J[2][3].
 * With w' = R_mu w, z = w'_z and theta = acos z, Eq. (log) is
 * nu = w'_xy * g(z) with g = theta / sin(theta), so
 *   d nu / d w' = [[g, 0, w'_x g'(z)], [0, g, w'_y g'(z)]],
 *   g'(z) = (theta cos theta - sin theta) / sin^3 theta  (limit -1/3 at z=1).
 * App. A prints a third column that does not satisfy J_log J_exp = I; this is
 * the derivative of the printed Eq. (log).
 */
void or_jlog(const double mu[3], const double w[3], double J[6])
{
    double R[9];
    or_basis(mu, R);
    double u = R[0] * w[0] + R[1] * w[1] + R[2] * w[2];
    double v = R[3] * w[0] + R[4] * w[1] + R[5] * w[2];
    double z = R[6] * w[0] + R[7] * w[1] + R[8] * w[2];
    double sn = sqrt(u * u + v * v);
    double th = atan2(sn, z);
    double g, gp;
    if (th < 1e-3) {
        double t2 = th * th;
        g = 1.0 + t2 / 6.0 + 7.0 * t2 * t2 / 360.0;
        gp = -1.0 / 3.0 - 2.0 * t2 / 15.0;  /* series of g'(z) in theta */
    } else {
        double st = sin(th);
        g = th / st;
        gp = (th * cos(th) - st) / (st * st * st);
    }
    double Jp[6] = { g, 0.0, u * gp, 0.0, g, v * gp };
    for (int row = 0; row < 2; ++row)
        for (int col = 0; col < 3; ++col)
            J[row * 3 + col] = Jp[row * 3 + 0] * R[0 * 3 + col] +
                               Jp[row * 3 + 1] * R[1 * 3 + col] +
                               Jp[row * 3 + 2] * R[2 * 3 + col];
}

/*
 * Textbook Cholesky of a 5x5 symmetric matrix given as a packed lower
 * triangle.  Returns 1 if the matrix is not positive definite.
 */
int or_cholesky5(const double S[15], double L[15])
{
#define P(i, j) ((i) * ((i) + 1) / 2 + (j))
    for (int j = 0; j < 5; ++j) {
        double d = S[P(j, j)];
        for (int p = 0; p < j; ++p) d -= L[P(j, p)] * L[P(j, p)];
        if (!(d > 0.0) || !isfinite(d)) return 1;
        L[P(j, j)] = sqrt(d);
        for (int i = j + 1; i < 5; ++i) {
            double e = S[P(i, j)];
            for (int p = 0; p < j; ++p) e -= L[P(i, p)] * L[P(j, p)];
            L[P(i, j)] = e / L[P(j, j)];
        }
    }
    return 0;
#undef P
}
