// query.cu -- conditioning, guided sampling and pdf of region mixtures on
// sm_103a (Sec. 3.1 "Density evaluation" and "Sampling", Sec. 3.2 closed-form
// conditioning, Sec. 3.3 one region's K components per query).
//
// A warp takes 32 queries at a time: lane l loads query l's position, region
// (array or grid) and uniforms (Philox or given) coalesced.  The queries are
// then processed SPI = 32/KP at a time with one lane per component (KP lanes
// per query), the query's inputs broadcast by shuffles; the component's
// query record stays in registers while consecutive queries share a region.
#include "common.cuh"
#include "kernels.h"

namespace sdmm {

template <int KP, int OP>
__global__ void __launch_bounds__(256)
    k_query(const float* __restrict__ qtab, int K, int64_t R, int64_t Q,
            const float* __restrict__ qx, const int32_t* __restrict__ region, GridF grid,
            uint64_t seed, const float* __restrict__ uni, const float* __restrict__ dir_in,
            float* __restrict__ cond_pi, float* __restrict__ cond_m, float* __restrict__ cond_L,
            float* __restrict__ dir_out, float* __restrict__ pdf_out,
            uint8_t* __restrict__ valid_out) {
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
                    int v = (int)floorf((xs[c] - grid.lo[c]) * grid.scale[c]);
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
                    const uint4 o = philox4x32_10(
                        make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 0u),
                        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
                    a0 = u24(o.x);
                    a1 = u24(o.y);
                    a2 = u24(o.z);
                }
            } else if (OP == OP_PDF) {
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
            float b0 = 0.f, b1 = 0.f, b2 = 0.f;
            if (OP != OP_CONDITION) {
                b0 = __shfl_sync(FULL, a0, src);
                b1 = __shfl_sync(FULL, a1, src);
                b2 = __shfl_sync(FULL, a2, src);
            }
            const bool ok = act && r >= 0;
            const int rl = r >= 0 ? r : 0;
            // ---- this lane's component record (reused while the region repeats)
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
                    P[11] = 1.f;
                    P[24] = P[26] = P[27] = P[29] = 1.f;
                    P[30] = -INFINITY;
                }
            }
            // ---- conditioning on position: z = A^-1 (x - mu^x)
            const float e0 = (qx0 - P[0]) - P[32], e1 = (qx1 - P[1]) - P[33],
                        e2 = (qx2 - P[2]) - P[34];
            const float z0 = P[12] * e0;
            const float z1 = P[13] * e0 + P[14] * e1;
            const float z2 = P[15] * e0 + P[16] * e1 + P[17] * e2;
            const float lw = P[30] - 0.5f * (z0 * z0 + z1 * z1 + z2 * z2);
            const float m0 = P[18] * z0 + P[19] * z1 + P[20] * z2;   // C^T z
            const float m1 = P[21] * z0 + P[22] * z1 + P[23] * z2;
            // normalise pi'_k over the KP component lanes (log-sum-exp)
            float mx = lw;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
            const float e = (mx == -INFINITY) ? 0.f : __expf(lw - mx);
            float se = e;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) se += __shfl_xor_sync(FULL, se, o);
            const float cpi = se > 0.f ? __fdividef(e, se) : 0.f;
            const int64_t qi = g + j;

            if (OP == OP_CONDITION) {
                if (act && k < K) {
                    const int64_t o = qi * K + k;
                    cond_pi[o] = ok ? cpi : 0.f;
                    cond_m[2 * o] = m0;
                    cond_m[2 * o + 1] = m1;
                    cond_L[3 * o] = P[24];
                    cond_L[3 * o + 1] = P[25];
                    cond_L[3 * o + 2] = P[26];
                }
                continue;
            }

            float w0 = b0, w1 = b1, w2 = b2;   // direction to evaluate
            int valid = 1;
            if (OP == OP_SAMPLE) {
                // component by inverse CDF on u0 (Sec. 3.1 "Sampling", step i)
                float cum = e;
#pragma unroll
                for (int o = 1; o < KP; o <<= 1) {
                    const float v = __shfl_up_sync(FULL, cum, o);
                    if (k >= o) cum += v;
                }
                const float tot = __shfl_sync(FULL, cum, base_lane + KP - 1);
                const float thr = b0 * tot;
                const unsigned seg = (KP == 32) ? FULL : (((1u << KP) - 1u) << base_lane);
                const unsigned hit = __ballot_sync(FULL, k < K && thr < cum) & seg;
                const unsigned pos = __ballot_sync(FULL, k < K && e > 0.f) & seg;
                int kk;
                if (hit) kk = __ffs(hit) - 1 - base_lane;
                else kk = pos ? (31 - __clz(pos)) - base_lane : 0;
                // Gaussian draw in the chart (step ii), exp map (step iii)
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, vv = 0.f;
                if (k == kk) {
                    const float rad = sqrtf(-2.f * logf(1.f - b1));
                    float sn, cs;
                    sincospif(2.f * b2, &sn, &cs);
                    const float g0 = rad * cs, g1 = rad * sn;
                    const float n0 = m0 + P[24] * g0;
                    const float n1 = m1 + P[25] * g0 + P[26] * g1;
                    const float rn = sqrtf(n0 * n0 + n1 * n1);
                    vv = rn < kPiF ? 1.f : 0.f;
                    float sr, cr;
                    sincosf(rn, &sr, &cr);
                    const float sc = rn < 1e-3f ? 1.f - rn * rn * (1.f / 6.f) : __fdividef(sr, rn);
                    const float c0 = n0 * sc, c1 = n1 * sc;
                    s0 = c0 * P[3] + c1 * P[6] + cr * P[9];
                    s1 = c0 * P[4] + c1 * P[7] + cr * P[10];
                    s2 = c0 * P[5] + c1 * P[8] + cr * P[11];
                }
                const int from = base_lane + kk;
                w0 = __shfl_sync(FULL, s0, from);
                w1 = __shfl_sync(FULL, s1, from);
                w2 = __shfl_sync(FULL, s2, from);
                valid = __shfl_sync(FULL, vv, from) > 0.5f && ok && pos != 0u;
            }
            // ---- solid-angle pdf of the conditioned mixture at w (Eq. solidangle-pdf)
            const float u = P[3] * w0 + P[4] * w1 + P[5] * w2;
            const float v = P[6] * w0 + P[7] * w1 + P[8] * w2;
            const float cz = P[9] * w0 + P[10] * w1 + P[11] * w2;
            const float s2v = u * u + v * v;
            const bool cut = s2v == 0.f && cz < 0.f;          // antipode: outside the chart
            const float gg = cut ? 1.f : g_of_cos(cz, rsqrtf(s2v));   // theta / sin(theta) = 1/sinc
            const float d0 = gg * u - m0, d1 = gg * v - m1;
            const float y0 = P[27] * d0;
            const float y1 = P[28] * d0 + P[29] * d1;
            float pk_ = cpi * __expf(P[31] - 0.5f * (y0 * y0 + y1 * y1)) * gg;
            if (cut || k >= K) pk_ = 0.f;
            float p = pk_;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) p += __shfl_xor_sync(FULL, p, o);
            if (act && k == 0) {
                if (OP == OP_SAMPLE) {
                    dir_out[3 * qi] = w0;
                    dir_out[3 * qi + 1] = w1;
                    dir_out[3 * qi + 2] = w2;
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
static cudaError_t launch_query_op(int KP, cudaStream_t s, int grid, const float* qtab, int K,
                                   int64_t R, int64_t Q, const float* qx, const int32_t* region,
                                   const GridF& g, uint64_t seed, const float* uni,
                                   const float* dir_in, float* cpi, float* cm, float* cL,
                                   float* dout, float* pout, uint8_t* vout) {
#define SDMM_Q_CASE(P)                                                                      \
    case P:                                                                                 \
        k_query<P, OP><<<grid, 256, 0, s>>>(qtab, K, R, Q, qx, region, g, seed, uni, dir_in, \
                                            cpi, cm, cL, dout, pout, vout);                 \
        break;
    switch (KP) {
        SDMM_Q_CASE(1)
        SDMM_Q_CASE(2)
        SDMM_Q_CASE(4)
        SDMM_Q_CASE(8)
        SDMM_Q_CASE(16)
        SDMM_Q_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef SDMM_Q_CASE
    return cudaGetLastError();
}

cudaError_t launch_query(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K,
                         int64_t R, int64_t Q, const float* qx, const int32_t* region,
                         const GridF& g, uint64_t seed, const float* uni, const float* dir_in,
                         float* cond_pi, float* cond_m, float* cond_L, float* dir_out,
                         float* pdf_out, uint8_t* valid_out) {
    switch (op) {
        case OP_CONDITION:
            return launch_query_op<OP_CONDITION>(KP, s, grid, qtab, K, R, Q, qx, region, g, seed,
                                                 uni, dir_in, cond_pi, cond_m, cond_L, dir_out,
                                                 pdf_out, valid_out);
        case OP_SAMPLE:
            return launch_query_op<OP_SAMPLE>(KP, s, grid, qtab, K, R, Q, qx, region, g, seed, uni,
                                              dir_in, cond_pi, cond_m, cond_L, dir_out, pdf_out,
                                              valid_out);
        default:
            return launch_query_op<OP_PDF>(KP, s, grid, qtab, K, R, Q, qx, region, g, seed, uni,
                                           dir_in, cond_pi, cond_m, cond_L, dir_out, pdf_out,
                                           valid_out);
    }
}

}  // namespace sdmm
