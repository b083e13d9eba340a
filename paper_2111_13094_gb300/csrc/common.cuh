// common.cuh -- device-side building blocks shared by the SDMM kernels:
// packed-triangle indexing, the chart rotation R_mu, the FP64 exp map and
// Jacobian used by the M-step, and the layout of the derived FP32 records.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmm.h"

namespace sdmm {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kLog2Pi = 1.8378770664093454835606594728112;
constexpr float kPiF = 3.14159265358979323846f;
// inverse CDF of the chi-square distribution with 3 dof at 0.9 (App. B)
constexpr double kChi2_3_q90 = 6.2513886311703222;

// entry (i, j <= i) of a packed lower-triangular 5x5 matrix
__host__ __device__ constexpr int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// Statistics per component in the work-unit partials: [s0, s1(5), s2(15)]
constexpr int kStat = 21;
// Shared per-sample features of the contraction form:
// [1, x' (3), vech(x'x') (6), w (3), w (x) x' (9), vech(ww) (6)]
constexpr int kFeat = 28;
// partial record of one work unit: K*21 component values, then W and sum w*l
__host__ __device__ inline int partial_stride(int K) { return ((K * kStat + 2) + 3) & ~3; }

// ---- derived FP32 records -------------------------------------------------
// E-step record (SDMM_ETAB_FLOATS = 36 floats):
//   [0..2] mu_x (+ position offset), rounded to FP32  [3..5] t  [6..8] b
//   [9..11] mu_w  [12..26] L^-1 packed
//   [27] c5 = log pi - sum log L_jj - (5/2) log 2 pi
//   [28..29] in-chart direction offset (0 except for objective evaluation)
//   [32..34] FP32 remainder of mu_x: x - mu = (x - hi) - lo keeps the
//            spatial difference accurate for narrow spatial components
// Query record (SDMM_QTAB_FLOATS = 36 floats), in two groups of whole float4:
// what conditioning on the position reads (float4 0-4), then what the pdf in
// the component's chart and the draw read (float4 5-8):
//   [0..2] mu_x (FP32)  [3] cx = log pi - log det A - (3/2) log 2 pi
//   [4..6] FP32 remainder of mu_x  [7..12] A^-1 packed  [13..18] C^T (2x3
//   row-major)  [19] 0  [20..22] t  [23..25] b  [26..28] mu_w
//   [29..31] D^-1  [32] cn = -log det D - log 2 pi  [33..35] D (d00, d10, d11)
// with L = [[A, 0], [C^T, D]] in (x, nu) order.
constexpr int kE = SDMM_ETAB_FLOATS;
constexpr int kQ = SDMM_QTAB_FLOATS;
namespace qrec {
constexpr int MUX = 0, CX = 3, REM = 4, AINV = 7, CT = 13, T = 20, B = 23, MUW = 26, DINV = 29, CN = 32, D = 33;
}

// R_mu with rows (t, b, mu): branchless orthonormal basis of Duff et al.,
// "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017.
__device__ inline void basis_f64(const double mu[3], double t[3], double b[3]) {
    const double sgn = copysign(1.0, mu[2]);
    const double a = -1.0 / (sgn + mu[2]);
    const double c = mu[0] * mu[1] * a;
    t[0] = 1.0 + sgn * mu[0] * mu[0] * a;
    t[1] = sgn * c;
    t[2] = -sgn * mu[0];
    b[0] = c;
    b[1] = sgn + mu[1] * mu[1] * a;
    b[2] = -mu[1];
}

// sin(r)/r with its Taylor series near zero
__device__ inline double sinc_f64(double r) {
    if (fabs(r) < 1e-4) {
        const double r2 = r * r;
        return 1.0 - r2 / 6.0 + r2 * r2 / 120.0;
    }
    return sin(r) / r;
}

// exp_mu(nu) = R_mu^T (nu sinc|nu|, cos|nu|)   (Sec. 3.1, Eq. exp)
__device__ inline void exp_map_f64(const double mu[3], const double nu[2], double out[3]) {
    double t[3], b[3];
    basis_f64(mu, t, b);
    const double r = sqrt(nu[0] * nu[0] + nu[1] * nu[1]);
    const double s = sinc_f64(r);
    const double a0 = nu[0] * s, a1 = nu[1] * s, a2 = cos(r);
    for (int c = 0; c < 3; ++c) out[c] = t[c] * a0 + b[c] * a1 + mu[c] * a2;
}

// New mean mu_new = exp_{mu_old}(nu) and the chart-change Jacobian
// J = J_log_{mu_new}(mu_new) * J_exp_{mu_old}(nu) (App. A; at the chart centre
// J_log is the projection onto (t, b) of mu_new), sharing one sincos.
__device__ inline void exp_map_jacobian_f64(const double mu_old[3], const double nu[2], double mu_new[3],
                                            double J[4]) {
    double t0[3], b0[3], t1[3], b1[3];
    basis_f64(mu_old, t0, b0);
    const double r2 = nu[0] * nu[0] + nu[1] * nu[1];
    const double r = sqrt(r2);
    double sr, cr;
    sincos(r, &sr, &cr);
    double s, c;
    if (r < 1e-2) {
        s = 1.0 - r2 / 6.0 + r2 * r2 / 120.0;
        c = -1.0 / 3.0 + r2 / 30.0 - r2 * r2 / 840.0;
    } else {
        const double ir = 1.0 / r;
        s = sr * ir;
        c = (cr - s) * (ir * ir);
    }
    const double a0 = nu[0] * s, a1 = nu[1] * s;
    for (int q = 0; q < 3; ++q) mu_new[q] = t0[q] * a0 + b0[q] * a1 + mu_old[q] * cr;
    basis_f64(mu_new, t1, b1);
    const double Jp[3][2] = {{s + nu[0] * nu[0] * c, nu[0] * nu[1] * c},
                             {nu[0] * nu[1] * c, s + nu[1] * nu[1] * c},
                             {-nu[0] * s, -nu[1] * s}};
    double Jw[3][2];
    for (int row = 0; row < 3; ++row)
        for (int col = 0; col < 2; ++col)
            Jw[row][col] = t0[row] * Jp[0][col] + b0[row] * Jp[1][col] + mu_old[row] * Jp[2][col];
    for (int col = 0; col < 2; ++col) {
        J[0 * 2 + col] = t1[0] * Jw[0][col] + t1[1] * Jw[1][col] + t1[2] * Jw[2][col];
        J[1 * 2 + col] = b1[0] * Jw[0][col] + b1[1] * Jw[1][col] + b1[2] * Jw[2][col];
    }
}

// atan2(s, c) for s >= 0, in [0, pi].  Octant reduction to t = min/max in
// [0, 1] and atan(t) = t P(t^2), P of degree 7 with coefficients fitted by
// csrc/fit_atan_poly.py (max relative error 2.2e-7 in FP32).
__device__ __forceinline__ float atan2_pos(float s, float c) {
    const float ac = fabsf(c);
    const float mn = fminf(s, ac), mx = fmaxf(s, ac);
    const float t = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float u = t * t;
    float p = -0.00482251868f;
    p = fmaf(p, u, 0.0247340072f);
    p = fmaf(p, u, -0.0602030531f);
    p = fmaf(p, u, 0.0996846780f);
    p = fmaf(p, u, -0.140413254f);
    p = fmaf(p, u, 0.199742138f);
    p = fmaf(p, u, -0.333323926f);
    p = fmaf(p, u, 1.0f) * t;
    if (s > ac) p = 1.57079637f - p;
    if (c < 0.f) p = 3.14159274f - p;
    return p;
}

// g = theta / sin(theta) of a unit direction from c = cos(theta) and
// rs = 1 / sin(theta), without the angle: g = P(1 - c) for c >= 0 and, since
// acos(c) = pi - acos(-c), g = pi rs - P(1 - |c|) for c < 0.  P(t) = 1 + ...
// of degree 9 fitted by csrc/fit_g_poly.py (max relative error 9.5e-8 in FP32
// on t in [0, 1]; 3.4e-7 for c < 0, just past pi / 2 where pi rs - P halves).  At the cut locus (rs infinite, c < 0) the result is
// infinite; callers treat that direction separately.
__device__ __forceinline__ float g_of_cos(float c, float rs) {
    const float t = 1.f - fabsf(c);
    float p = 0.0111601921f;
    p = fmaf(p, t, -0.0325264037f);
    p = fmaf(p, t, 0.0507297404f);
    p = fmaf(p, t, -0.0331454873f);
    p = fmaf(p, t, 0.029695496f);
    p = fmaf(p, t, 0.0203489829f);
    p = fmaf(p, t, 0.0579242408f);
    p = fmaf(p, t, 0.133274719f);
    p = fmaf(p, t, 0.333334833f);
    p = fmaf(p, t, 1.0f);
    return c < 0.f ? fmaf(3.14159274f, rs, -p) : p;
}

// The same g = theta / sin(theta) with a degree-7 P (csrc/fit_g_poly.py 7: max
// relative error 5.4e-7 in FP32), for the E-step of the fit: there g scales
// the chart coordinates of every (sample, component) pair, an error of 5.4e-7
// moves a log-likelihood by that fraction of its directional Mahalanobis
// term, far inside the 1e-4 parity of the fit, and costs two fused
// multiply-adds less.  Queries keep the degree-9 form (their pdf parity is
// 1e-5).
__device__ __forceinline__ float g_of_cos_fit(float c, float rs) {
    const float t = 1.f - fabsf(c);
    float p = 0.0264989268f;
    p = fmaf(p, t, -0.0498756915f);
    p = fmaf(p, t, 0.0664620921f);
    p = fmaf(p, t, -0.0025986f);
    p = fmaf(p, t, 0.0645030662f);
    p = fmaf(p, t, 0.132436037f);
    p = fmaf(p, t, 0.333369762f);
    p = fmaf(p, t, 1.0f);
    return c < 0.f ? fmaf(3.14159274f, rs, -p) : p;
}

// Cholesky of a packed symmetric 5x5; false if not positive definite.
__device__ inline bool cholesky5_f64(const double S[15], double L[15]) {
    for (int j = 0; j < 5; ++j) {
        double d = S[pk(j, j)];
        for (int p = 0; p < j; ++p) d -= L[pk(j, p)] * L[pk(j, p)];
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double ljj = sqrt(d);
        const double il = 1.0 / ljj;
        L[pk(j, j)] = ljj;
        for (int i = j + 1; i < 5; ++i) {
            double e = S[pk(i, j)];
            for (int p = 0; p < j; ++p) e -= L[pk(i, p)] * L[pk(j, p)];
            L[pk(i, j)] = e * il;
        }
    }
    return true;
}

// Inverse of a packed lower-triangular 5x5 (also lower triangular).
__device__ inline void lower_inverse5_f64(const double L[15], double Li[15]) {
    for (int j = 0; j < 5; ++j) Li[pk(j, j)] = 1.0 / L[pk(j, j)];
    for (int j = 0; j < 5; ++j) {
        for (int i = j + 1; i < 5; ++i) {
            double s = 0.0;
            for (int p = j; p < i; ++p) s += L[pk(i, p)] * Li[pk(p, j)];
            Li[pk(i, j)] = -s * Li[pk(i, i)];
        }
    }
}

// Writes the E-step and query records of one component.
__device__ inline void write_records(double pi, const double mux[3], const double muw[3],
                                     const double L[15], float* __restrict__ er,
                                     float* __restrict__ qr, const double* delta = nullptr,
                                     bool euclid = false) {
    double t[3], b[3], Li[15];
    if (euclid) {   // nu = (w_x, w_y) - (mu_x, mu_y): unit rows, the mean as the offset
        t[0] = 1.0, t[1] = 0.0, t[2] = 0.0;
        b[0] = 0.0, b[1] = 1.0, b[2] = 0.0;
    } else {
        basis_f64(muw, t, b);
    }
    lower_inverse5_f64(L, Li);
    const double lpi = pi > 0.0 ? log(pi) : -INFINITY;
    // log det of the blocks as the log of the product of the pivots (two FP64
    // logs instead of five; the pivots are far from the FP64 range's ends)
    const double ldA = log(L[pk(0, 0)] * L[pk(1, 1)] * L[pk(2, 2)]);
    const double ldD = log(L[pk(3, 3)] * L[pk(4, 4)]);
    for (int c = 0; c < 3; ++c) {
        er[0 + c] = qr[qrec::MUX + c] = (float)mux[c];
        er[3 + c] = qr[qrec::T + c] = (float)t[c];
        er[6 + c] = qr[qrec::B + c] = (float)b[c];
        er[9 + c] = qr[qrec::MUW + c] = (float)muw[c];
    }
    for (int p = 0; p < 15; ++p) er[12 + p] = (float)Li[p];
    er[27] = (float)(lpi - ldA - ldD - 2.5 * kLog2Pi);
    er[28] = er[29] = er[30] = er[31] = er[35] = qr[19] = 0.f;
    double me[3] = {mux[0], mux[1], mux[2]};
    if (delta != nullptr) {
        for (int c = 0; c < 3; ++c) me[c] += delta[c];
        er[28] = (float)delta[3];
        er[29] = (float)delta[4];
    }
    if (euclid) {
        er[28] = (float)(muw[0] + (delta != nullptr ? delta[3] : 0.0));
        er[29] = (float)(muw[1] + (delta != nullptr ? delta[4] : 0.0));
    }
    for (int c = 0; c < 3; ++c) {
        er[c] = (float)me[c];
        er[32 + c] = (float)(me[c] - (double)er[c]);
        qr[qrec::REM + c] = (float)(mux[c] - (double)qr[qrec::MUX + c]);
    }
    for (int p = 0; p < 6; ++p) qr[qrec::AINV + p] = (float)Li[p];
    for (int c = 0; c < 3; ++c) {
        qr[qrec::CT + c] = (float)L[pk(3, c)];
        qr[qrec::CT + 3 + c] = (float)L[pk(4, c)];
    }
    qr[qrec::D + 0] = (float)L[pk(3, 3)];
    qr[qrec::D + 1] = (float)L[pk(4, 3)];
    qr[qrec::D + 2] = (float)L[pk(4, 4)];
    qr[qrec::DINV + 0] = (float)Li[pk(3, 3)];
    qr[qrec::DINV + 1] = (float)Li[pk(4, 3)];
    qr[qrec::DINV + 2] = (float)Li[pk(4, 4)];
    qr[qrec::CX] = (float)(lpi - ldA - 1.5 * kLog2Pi);
    qr[qrec::CN] = (float)(-ldD - kLog2Pi);
}

// Batch descriptor written into the workspace before each fit step sequence.
struct BatchDesc {
    const float* p[7];          // px py pz ox oy oz w
    const int64_t* offsets;
    int64_t R;
    int64_t N;
    const double* prior_scale;  // nullable
    float* loglik;              // nullable
};

// Workspace header (device)
struct WsHeader {
    BatchDesc desc;
    int32_t n_chunks;
    int32_t queue;
    int32_t err;        // set by the tensor-core E-step when an MMA wait times out
    int32_t pad_[13];
};

// Philox4x32-10: J. K. Salmon et al., "Parallel Random Numbers: As Easy as
// 1, 2, 3", SC'11.  Ten rounds of two 32x32->64 multiplies mixed with the other
// counter words and a Weyl-sequence key.
__device__ inline uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i > 0) {
            k.x += W0;
            k.y += W1;
        }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ inline float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

}  // namespace sdmm
