// product.cu -- product sampling of a region's conditioned radiance mixture
// with a small BSDF mixture (Sec. 3.5 "Product Sampling from Mixed-
// Orientation Gaussians", Eq. product-distribution; Sec. 4.1 "Pruning before
// product sampling"), FP32.
//
// Layout as in k_query: KP lanes per query, lane k = radiance component k
// (its query record in registers), SPI = 32/KP queries per warp step.  After
// conditioning on the position, lane k forms its pairs with the two BSDF
// lobes of largest weight: in the chart of mu_k the lobe has mean
// nu2 = log_{mu_k}(mu2) and covariance J S2 J^T, J = J_log_{mu_k}(mu2)
// J_exp_{mu2}(0); the product of N(m_k, S1) and N(nu2, S2') is a Gaussian
// (P = S1 (S1+S2')^-1 S2', mean S2' (S1+S2')^-1 m_k + S1 (S1+S2')^-1 nu2)
// weighted by pi'_k w_j N(m_k; nu2, S1 + S2').  Pairs are ordered by
// component, then lobe index; sampling picks one by inverse CDF over the
// lanes, draws in its chart and maps with exp; the pdf on the sphere sums
// every pair's chart density divided by sinc.
#include "common.cuh"
#include "kernels.h"

namespace sdmm {

constexpr float kTwoPiF = 6.28318530717958647692f;

// Duff et al.'s branchless basis (rows t, b of R_mu), FP32
__device__ __forceinline__ void basis_f32(float m0, float m1, float m2, float t[3], float b[3]) {
    const float sgn = copysignf(1.f, m2);
    const float a = __fdividef(-1.f, sgn + m2);
    const float c = m0 * m1 * a;
    t[0] = 1.f + sgn * m0 * m0 * a;
    t[1] = sgn * c;
    t[2] = -sgn * m0;
    b[0] = c;
    b[1] = sgn + m1 * m1 * a;
    b[2] = -m1;
}

// One (component, lobe) pair in the component's chart: the product's
// Cholesky factor C = [[1/i0, 0], [p10, 1/i1]] (kept as reciprocal diagonals),
// mean and log weight (log pi' + log w + log N(m; nu2, S1 + S2')).
struct Pair {
    float m0, m1, i0, p10, i1, ln, lw;
};

__device__ inline Pair make_pair(const float* P, float cm0, float cm1, float lcpi, float wj, const float* mu2,
                                 const float* L2) {
    Pair o;
    o.m0 = o.m1 = 0.f;
    o.i0 = o.i1 = 1.f;
    o.p10 = o.ln = 0.f;
    o.lw = -INFINITY;
    // the lobe's mean in the mu_k chart
    const float u = P[qrec::T] * mu2[0] + P[qrec::T + 1] * mu2[1] + P[qrec::T + 2] * mu2[2];
    const float v = P[qrec::B] * mu2[0] + P[qrec::B + 1] * mu2[1] + P[qrec::B + 2] * mu2[2];
    const float c = P[qrec::MUW] * mu2[0] + P[qrec::MUW + 1] * mu2[1] + P[qrec::MUW + 2] * mu2[2];
    const float s2 = u * u + v * v;
    const float rs = rsqrtf(s2);
    const float s = s2 > 0.f ? s2 * rs : 0.f;
    const float th = atan2_pos(s, c);
    if ((s2 == 0.f && c < 0.f) || th >= kPiF || !(wj > 0.f)) return o;   // antipode / no weight
    const float g = s2 > 0.f ? th * rs : 1.f;
    // d g / d c along the sphere: (theta c - s) / s^3, its series below 0.05 rad
    const float h = th < 0.05f ? -1.f / 3.f - (2.f / 15.f) * th * th : (th * c - s) * (rs * rs * rs);
    const float n0 = g * u, n1 = g * v;
    // J = J_log(mu2) [t2 b2]: tangent directions of the lobe's chart seen in the mu_k chart
    float t2[3], b2[3];
    basis_f32(mu2[0], mu2[1], mu2[2], t2, b2);
    float J[2][2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float e0 = q == 0 ? t2[0] : b2[0], e1 = q == 0 ? t2[1] : b2[1], e2 = q == 0 ? t2[2] : b2[2];
        const float ta = P[qrec::T] * e0 + P[qrec::T + 1] * e1 + P[qrec::T + 2] * e2;
        const float tb = P[qrec::B] * e0 + P[qrec::B + 1] * e1 + P[qrec::B + 2] * e2;
        const float tc = P[qrec::MUW] * e0 + P[qrec::MUW + 1] * e1 + P[qrec::MUW + 2] * e2;
        J[0][q] = g * ta + u * tc * h;
        J[1][q] = g * tb + v * tc * h;
    }
    // S2' = (J L2)(J L2)^T, S1 = D D^T
    const float M00 = J[0][0] * L2[0] + J[0][1] * L2[1], M01 = J[0][1] * L2[2];
    const float M10 = J[1][0] * L2[0] + J[1][1] * L2[1], M11 = J[1][1] * L2[2];
    const float b00 = M00 * M00 + M01 * M01, b01 = M00 * M10 + M01 * M11, b11 = M10 * M10 + M11 * M11;
    const float d00 = P[qrec::D], d10 = P[qrec::D + 1], d11 = P[qrec::D + 2];
    const float a00 = d00 * d00, a01 = d00 * d10, a11 = d10 * d10 + d11 * d11;
    // S = S1 + S2' and its inverse
    const float S00 = a00 + b00, S01 = a01 + b01, S11 = a11 + b11;
    const float det = S00 * S11 - S01 * S01;
    if (!(det > 0.f)) return o;
    const float id = __fdividef(1.f, det);
    const float i00 = S11 * id, i01 = -S01 * id, i11 = S00 * id;
    const float d0 = cm0 - n0, d1 = cm1 - n1;
    const float q = d0 * (i00 * d0 + i01 * d1) + d1 * (i01 * d0 + i11 * d1);
    o.lw = lcpi - 0.5f * q - __logf(kTwoPiF) + __logf(wj * rsqrtf(det));
    // P = S1 Si S2', mean = S2' Si m + S1 Si nu2
    const float X00 = i00 * b00 + i01 * b01, X01 = i00 * b01 + i01 * b11;   // Si S2'
    const float X10 = i01 * b00 + i11 * b01, X11 = i01 * b01 + i11 * b11;
    const float P00 = a00 * X00 + a01 * X10, P11 = a01 * X01 + a11 * X11;
    const float P01 = 0.5f * ((a00 * X01 + a01 * X11) + (a01 * X00 + a11 * X10));
    const float y0 = i00 * cm0 + i01 * cm1, y1 = i01 * cm0 + i11 * cm1;      // Si m
    const float z0 = i00 * n0 + i01 * n1, z1 = i01 * n0 + i11 * n1;          // Si nu2
    o.m0 = b00 * y0 + b01 * y1 + a00 * z0 + a01 * z1;
    o.m1 = b01 * y0 + b11 * y1 + a01 * z0 + a11 * z1;
    o.i0 = rsqrtf(P00);
    o.p10 = P01 * o.i0;
    o.i1 = rsqrtf(fmaxf(P11 - o.p10 * o.p10, 1e-30f));
    o.ln = __logf(o.i0 * o.i1) - __logf(kTwoPiF);
    return o;
}

// log of the pair's chart density at nu (without the weight)
__device__ __forceinline__ float pair_logpdf(const Pair& p, float nu0, float nu1) {
    const float y0 = (nu0 - p.m0) * p.i0;
    const float y1 = (nu1 - p.m1 - p.p10 * y0) * p.i1;
    return p.ln - 0.5f * (y0 * y0 + y1 * y1);
}

template <int KP, int OP>
__global__ void __launch_bounds__(256, 3)
    k_product(const float* __restrict__ qtab, int K, int64_t R, int64_t Q, const float* __restrict__ qx,
              const int32_t* __restrict__ region, GridF grid, const float* __restrict__ bw,
              const float* __restrict__ bmu, const float* __restrict__ bL, int J, uint64_t seed,
              const float* __restrict__ uni, const float* __restrict__ dir_in, float* __restrict__ dir_out,
              float* __restrict__ pdf_out, uint8_t* __restrict__ valid_out) {
    constexpr int SPI = 32 / KP;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int k = lane & (KP - 1), h = lane / KP, base_lane = h * KP;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

    float P[kQ];
    int cur_r = -1;
    for (int64_t g = gw * 32; g < Q; g += warps * 32) {
        // ---- per-lane query inputs, coalesced
        const int64_t i = g + lane;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
        int rr = -1;
        if (i < Q) {
            x0 = qx[3 * i];
            x1 = qx[3 * i + 1];
            x2 = qx[3 * i + 2];
            if (region != nullptr) {
                rr = region[i];
            } else {
                const float xs[3] = {x0, x1, x2};
                int id[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int v = (int)floorf((xs[c] - grid.lo[c]) * grid.scale[c]);
                    id[c] = min(max(v, 0), grid.dims[c] - 1);
                }
                rr = id[0] + grid.dims[0] * (id[1] + grid.dims[1] * id[2]);
            }
            if (rr < 0 || rr >= R) rr = -1;
            if (OP == OP_SAMPLE) {
                if (uni != nullptr) {
                    a0 = uni[3 * i];
                    a1 = uni[3 * i + 1];
                    a2 = uni[3 * i + 2];
                } else {
                    const uint4 o = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 0u),
                                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
                    a0 = u24(o.x);
                    a1 = u24(o.y);
                    a2 = u24(o.z);
                }
            } else {
                a0 = dir_in[3 * i];
                a1 = dir_in[3 * i + 1];
                a2 = dir_in[3 * i + 2];
            }
        }
        const int n = (int)min((int64_t)32, Q - g);
        for (int t = 0; t < n; t += SPI) {
            const int j = t + h;
            const bool act = j < n;
            const int src = act ? j : t;
            const float qx0 = __shfl_sync(FULL, x0, src), qx1 = __shfl_sync(FULL, x1, src),
                        qx2 = __shfl_sync(FULL, x2, src);
            const int r = __shfl_sync(FULL, rr, src);
            const float b0 = __shfl_sync(FULL, a0, src), b1 = __shfl_sync(FULL, a1, src),
                        b2 = __shfl_sync(FULL, a2, src);
            const bool ok = act && r >= 0;
            const int rl = r >= 0 ? r : 0;
            if (rl != cur_r) {
                cur_r = rl;
                if (k < K) {
                    const float4* s = reinterpret_cast<const float4*>(qtab + ((int64_t)rl * K + k) * kQ);
#pragma unroll
                    for (int q = 0; q < kQ / 4; ++q) {
                        const float4 v = __ldg(s + q);
                        P[4 * q] = v.x;
                        P[4 * q + 1] = v.y;
                        P[4 * q + 2] = v.z;
                        P[4 * q + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kQ; ++q) P[q] = 0.f;
                    P[qrec::MUW + 2] = 1.f;
                    P[qrec::D] = P[qrec::D + 2] = P[qrec::DINV] = P[qrec::DINV + 2] = 1.f;
                    P[qrec::CX] = -INFINITY;
                }
            }
            // ---- conditioning on position (as in k_query)
            const float e0 = (qx0 - P[qrec::MUX]) - P[qrec::REM];
            const float e1 = (qx1 - P[qrec::MUX + 1]) - P[qrec::REM + 1];
            const float e2 = (qx2 - P[qrec::MUX + 2]) - P[qrec::REM + 2];
            const float z0 = P[qrec::AINV] * e0;
            const float z1 = P[qrec::AINV + 1] * e0 + P[qrec::AINV + 2] * e1;
            const float z2 = P[qrec::AINV + 3] * e0 + P[qrec::AINV + 4] * e1 + P[qrec::AINV + 5] * e2;
            const float lw = P[qrec::CX] - 0.5f * (z0 * z0 + z1 * z1 + z2 * z2);
            const float m0 = P[qrec::CT] * z0 + P[qrec::CT + 1] * z1 + P[qrec::CT + 2] * z2;
            const float m1 = P[qrec::CT + 3] * z0 + P[qrec::CT + 4] * z1 + P[qrec::CT + 5] * z2;
            float mx = lw;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
            const float ec = (mx == -INFINITY) ? 0.f : __expf(lw - mx);
            float se = ec;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) se += __shfl_xor_sync(FULL, se, o);
            const float lcpi = (se > 0.f && ec > 0.f && k < K) ? (lw - mx) - __logf(se) : -INFINITY;   // log pi'_k
            // ---- the two BSDF lobes of largest weight, in increasing index
            const int64_t qi = g + j;
            const int64_t qb = ok ? qi : 0;
            int j1 = -1, j2 = -1;
            float w1 = -1.f, w2 = -1.f;
            for (int l = 0; l < J; ++l) {
                const float wl = __ldg(bw + qb * J + l);
                if (wl > w1) {
                    j2 = j1;
                    w2 = w1;
                    j1 = l;
                    w1 = wl;
                } else if (wl > w2) {
                    j2 = l;
                    w2 = wl;
                }
            }
            const int ja = (j2 >= 0 && j2 < j1) ? j2 : j1, jb = (j2 >= 0 && j2 < j1) ? j1 : j2;
            Pair pr[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int jl = q == 0 ? ja : jb;
                if (jl >= 0 && ok) {
                    float mu2[3], L2[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        mu2[c] = __ldg(bmu + (qb * J + jl) * 3 + c);
                        L2[c] = __ldg(bL + (qb * J + jl) * 3 + c);
                    }
                    pr[q] = make_pair(P, m0, m1, lcpi, __ldg(bw + qb * J + jl), mu2, L2);
                } else {
                    pr[q] = make_pair(P, m0, m1, -INFINITY, 0.f, P + qrec::MUW, P + qrec::D);   // no pair
                }
            }
            // ---- normalise the pair weights over the query's lanes
            float pm = fmaxf(pr[0].lw, pr[1].lw);
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) pm = fmaxf(pm, __shfl_xor_sync(FULL, pm, o));
            const float ea = pm == -INFINITY ? 0.f : __expf(pr[0].lw - pm);
            const float eb = pm == -INFINITY ? 0.f : __expf(pr[1].lw - pm);
            float tot = ea + eb;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);

            float w0 = b0, wv1 = b1, wv2 = b2;   // direction to evaluate
            int valid = 1;
            if (OP == OP_SAMPLE) {
                float cum = ea + eb;
#pragma unroll
                for (int o = 1; o < KP; o <<= 1) {
                    const float v = __shfl_up_sync(FULL, cum, o);
                    if (k >= o) cum += v;
                }
                const float thr = b0 * tot;
                const unsigned seg = (KP == 32) ? FULL : (((1u << KP) - 1u) << base_lane);
                const unsigned hit = __ballot_sync(FULL, thr < cum) & seg;
                const unsigned pos = __ballot_sync(FULL, ea + eb > 0.f) & seg;
                int kk;
                if (hit) kk = __ffs(hit) - 1 - base_lane;
                else kk = pos ? (31 - __clz(pos)) - base_lane : 0;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, vv = 0.f;
                if (k == kk) {
                    // inside the lane: pair a unless the threshold lies past it
                    const bool use_b = !(thr < cum - eb) || !(ea > 0.f);
                    const bool pb = use_b && eb > 0.f;
                    Pair p;
                    p.m0 = pb ? pr[1].m0 : pr[0].m0;
                    p.m1 = pb ? pr[1].m1 : pr[0].m1;
                    p.i0 = pb ? pr[1].i0 : pr[0].i0;
                    p.p10 = pb ? pr[1].p10 : pr[0].p10;
                    p.i1 = pb ? pr[1].i1 : pr[0].i1;
                    const float rad = sqrtf(-2.f * logf(1.f - b1));
                    float sn, cs;
                    sincospif(2.f * b2, &sn, &cs);
                    const float g0 = rad * cs, g1 = rad * sn;
                    const float z0 = __fdividef(g0, p.i0);
                    const float n0 = p.m0 + z0;
                    const float n1 = p.m1 + p.p10 * g0 + __fdividef(g1, p.i1);
                    const float rn = sqrtf(n0 * n0 + n1 * n1);
                    vv = rn < kPiF ? 1.f : 0.f;
                    float sr, cr;
                    sincosf(rn, &sr, &cr);
                    const float sc = rn < 1e-3f ? 1.f - rn * rn * (1.f / 6.f) : __fdividef(sr, rn);
                    const float c0 = n0 * sc, c1 = n1 * sc;
                    s0 = c0 * P[qrec::T] + c1 * P[qrec::B] + cr * P[qrec::MUW];
                    s1 = c0 * P[qrec::T + 1] + c1 * P[qrec::B + 1] + cr * P[qrec::MUW + 1];
                    s2 = c0 * P[qrec::T + 2] + c1 * P[qrec::B + 2] + cr * P[qrec::MUW + 2];
                }
                const int from = base_lane + kk;
                w0 = __shfl_sync(FULL, s0, from);
                wv1 = __shfl_sync(FULL, s1, from);
                wv2 = __shfl_sync(FULL, s2, from);
                valid = __shfl_sync(FULL, vv, from) > 0.5f && ok && pos != 0u;
            }
            // ---- pdf of the product mixture at w: every pair's chart density / sinc
            const float u = P[qrec::T] * w0 + P[qrec::T + 1] * wv1 + P[qrec::T + 2] * wv2;
            const float v = P[qrec::B] * w0 + P[qrec::B + 1] * wv1 + P[qrec::B + 2] * wv2;
            const float cz = P[qrec::MUW] * w0 + P[qrec::MUW + 1] * wv1 + P[qrec::MUW + 2] * wv2;
            const float s2v = u * u + v * v;
            const bool cut = s2v == 0.f && cz < 0.f;          // antipode: outside the chart
            const float gg = cut ? 1.f : g_of_cos(cz, rsqrtf(s2v));
            const float nu0 = gg * u, nu1 = gg * v;
            float pk = 0.f;
            if (!cut && k < K) {
                if (ea > 0.f) pk += ea * __expf(pair_logpdf(pr[0], nu0, nu1));
                if (eb > 0.f) pk += eb * __expf(pair_logpdf(pr[1], nu0, nu1));
                pk *= gg;
            }
            float p = pk;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) p += __shfl_xor_sync(FULL, p, o);
            p = tot > 0.f ? p / tot : 0.f;
            if (act && k == 0) {
                if (OP == OP_SAMPLE) {
                    dir_out[3 * qi] = w0;
                    dir_out[3 * qi + 1] = wv1;
                    dir_out[3 * qi + 2] = wv2;
                    valid_out[qi] = (uint8_t)valid;
                    pdf_out[qi] = valid ? p : 0.f;
                } else {
                    pdf_out[qi] = ok ? p : 0.f;
                }
            }
        }
    }
}

template <int OP>
static cudaError_t launch_product_op(int KP, cudaStream_t s, int grid, const float* qtab, int K, int64_t R,
                                     int64_t Q, const float* qx, const int32_t* region, const GridF& g,
                                     const float* bw, const float* bmu, const float* bL, int J, uint64_t seed,
                                     const float* uni, const float* dir_in, float* dout, float* pout,
                                     uint8_t* vout) {
#define SDMM_P_CASE(PP)                                                                                  \
    case PP:                                                                                             \
        k_product<PP, OP><<<grid, 256, 0, s>>>(qtab, K, R, Q, qx, region, g, bw, bmu, bL, J, seed, uni,  \
                                               dir_in, dout, pout, vout);                                \
        break;
    switch (KP) {
        SDMM_P_CASE(1)
        SDMM_P_CASE(2)
        SDMM_P_CASE(4)
        SDMM_P_CASE(8)
        SDMM_P_CASE(16)
        SDMM_P_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef SDMM_P_CASE
    return cudaGetLastError();
}

cudaError_t launch_product(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K, int64_t R, int64_t Q,
                           const float* qx, const int32_t* region, const GridF& g, const float* bw, const float* bmu,
                           const float* bL, int J, uint64_t seed, const float* uni, const float* dir_in, float* dout,
                           float* pout, uint8_t* vout) {
    if (op == OP_SAMPLE)
        return launch_product_op<OP_SAMPLE>(KP, s, grid, qtab, K, R, Q, qx, region, g, bw, bmu, bL, J, seed, uni,
                                            dir_in, dout, pout, vout);
    return launch_product_op<OP_PDF>(KP, s, grid, qtab, K, R, Q, qx, region, g, bw, bmu, bL, J, seed, uni, dir_in,
                                     dout, pout, vout);
}

}  // namespace sdmm
