// query.cu -- conditioning, guided sampling and pdf of region mixtures on
// sm_103a (Sec. 3.1 "Density evaluation" and "Sampling", Sec. 3.2 closed-form
// conditioning, Sec. 3.3 one region's K components per query).
//
// A warp takes 32 queries at a time: lane l loads query l's position, region
// (array or grid) and uniforms (Philox or given) coalesced.  The queries are
// then processed SPI = 32/KP at a time with one lane per component (KP lanes
// per query), the query's inputs broadcast by shuffles; the component's
// query record stays in registers while consecutive queries share a region.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace sdmm {

// ---------------------------------------------------------------------------
// Guided sampling and pdf with one thread per query (K <= KM components).
// The thread conditions every component of its region on the position in a
// first pass (weight and conditional mean of each component kept in shared
// memory, in a per-thread slot of two arrays), picks the component and draws
// the direction, then evaluates the solid-angle pdf of the conditioned mixture
// at that direction in a second pass.  No lane waits on another: the component
// choice, the Gaussian draw and the exp map run once per query instead of in
// one lane of a component group.
//
// With `perm` (the library's binning) query perm[j] is processed at slot j
// (perm[j] < 0: an empty padding slot) and its outputs go to the slot's record
// sorted_out[j]: (direction, pdf, or -1 if not valid) for sampling, (pdf, ...)
// for the pdf; k_qbin_unpermute then moves them to the query's own index.
// Without it, outputs go to the query's own index.
// Each warp of the persistent grid takes a contiguous run of batches of 32
// slots.  When a batch's queries fall in at most two regions, those of its
// first and last query (queries sorted by region), the warp copies a region's
// K records into shared memory with coalesced 16-byte loads, rescaled for the
// base-2 exponents (only when the region changes, so once per region for
// sorted queries), and the threads of that region read them from there, one
// pass per region.  A batch whose queries span more regions (queries in any
// order) is processed with one lane per component instead
// (warp_by_components), which reads each query's records once, coalesced.
constexpr int kQWarps = 4;

template <int KP, int OP>
__device__ __forceinline__ void warp_by_components(const float* __restrict__ qtab, int K, unsigned active, int64_t il,
                                                   float x0, float x1, float x2, int rr, float a0, float a1,
                                                   float a2, float* P, int& cur_r, float* __restrict__ cond_pi,
                                                   float* __restrict__ cond_m, float* __restrict__ cond_L,
                                                   float* __restrict__ dir_out, float* __restrict__ pdf_out,
                                                   uint8_t* __restrict__ valid_out, float4* __restrict__ sorted_out,
                                                   int64_t slot0);

constexpr int kQCtas = 5;        // resident CTAs per SM (registers and shared memory allow five)

template <int KM, int OP>
__global__ void __launch_bounds__(kQWarps * 32, kQCtas)
    k_query_q(const float* __restrict__ qtab, int K, int64_t R, int64_t Q,
              const float* __restrict__ qx, const int32_t* __restrict__ region, GridF grid,
              const int32_t* __restrict__ perm, float4* __restrict__ sorted_out, uint64_t seed,
              const float* __restrict__ uni, const float* __restrict__ dir_in, float* __restrict__ dir_out,
              float* __restrict__ pdf_out, uint8_t* __restrict__ valid_out) {
    static_assert(OP == OP_SAMPLE || OP == OP_PDF, "sampling and pdf only");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr float kL2e = 1.44269504088896341f;
    constexpr float kC = 0.849321800288019f;                   // sqrt(log2(e) / 2)
    constexpr float kIC = 1.177410022515475f;                  // 1 / kC
    constexpr int Q4 = kQ / 4;                                 // float4 per record
    __shared__ float4 s_rec[kQWarps][KM * Q4];                 // per warp: one region's records
    // per thread and component: the weight w'_k and the conditional mean m_k,
    // in separate arrays so that a warp's 32 weights are one conflict-free
    // wavefront (interleaved with the means they were four)
    __shared__ float s_cw[KM][kQWarps * 32];
    __shared__ float2 s_cmu[KM][kQWarps * 32];
    // per float4 of a record, the factors of its staged copy: A^-1 and D^-1
    // times c = sqrt(log2(e) / 2), C^T times 1 / c, cn times log2(e)
    __shared__ float4 s_scale[Q4];
    if (threadIdx.x < Q4) {
        const int m = threadIdx.x;
        float4 f = make_float4(1.f, 1.f, 1.f, 1.f);
        if (m == 1) f.w = kC;                                              // (rem, A^-1 0)
        if (m == 2) f = make_float4(kC, kC, kC, kC);                       // A^-1 1..4
        if (m == 3) f = make_float4(kC, kIC, kIC, kIC);                    // (A^-1 5, C^T 0)
        if (m == 4) f = make_float4(kIC, kIC, kIC, 1.f);                   // (C^T 1, 0)
        if (m == 7) f = make_float4(1.f, kC, kC, kC);                      // (mu_w.z, D^-1)
        if (m == 8) f.x = kL2e;                                            // (cn, D)
        s_scale[m] = f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* __restrict__ q4 = reinterpret_cast<const float4*>(qtab);
    const int n4 = K * Q4;                                     // float4 of one region's records
    float* const cw = &s_cw[0][threadIdx.x];                   // component k at cw[k * CS]
    float2* const cmu = &s_cmu[0][threadIdx.x];                // and cmu[k * CS]
    constexpr int CS = kQWarps * 32;
    int staged = -1;
    // each warp takes a contiguous run of batches of 32 slots, so that sorted
    // queries stage a region's records once per region, not once per batch
    const int64_t nbat = (Q + 31) / 32, nwarps = (int64_t)gridDim.x * kQWarps;
    const int64_t per = (nbat + nwarps - 1) / nwarps;
    const int64_t b0 = ((int64_t)blockIdx.x * kQWarps + warp) * per;
    const int64_t b1 = b0 + per < nbat ? b0 + per : nbat;
    for (int64_t bat = b0; bat < b1; ++bat) {
        const int64_t base = bat * 32;
        const int64_t j = base + lane;
        bool in = j < Q;
        int64_t i = j;
        int r = -1;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (in && perm != nullptr) {           // sorted positions; -1 marks padding
            i = perm[j];
            in = i >= 0;
        }
        if (in) {
            if (region != nullptr) r = region[i];
            x0 = qx[3 * i];
            x1 = qx[3 * i + 1];
            x2 = qx[3 * i + 2];
            if (region == nullptr) {
                const float xs[3] = {x0, x1, x2};
                int id[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int v = (int)floorf((xs[c] - grid.lo[c]) * grid.scale[c]);
                    id[c] = min(max(v, 0), grid.dims[c] - 1);
                }
                r = id[0] + grid.dims[0] * (id[1] + grid.dims[1] * id[2]);
            }
        }
        const bool ok = in && r >= 0 && r < R;
        const int rr = ok ? r : 0;
        const unsigned act = __ballot_sync(FULL, in);
        if (act == 0u) continue;
        const int r0 = __shfl_sync(FULL, rr, __ffs(act) - 1);   // region of the first query
        const int r1 = __shfl_sync(FULL, rr, 31 - __clz(act));  // and of the last
        if (!__all_sync(FULL, !in || rr == r0 || rr == r1)) {
            // queries of several regions (given in any order): one lane per
            // component, each query's records read once, coalesced
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
            if (in) {
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
                } else {
                    a0 = dir_in[3 * i];
                    a1 = dir_in[3 * i + 1];
                    a2 = dir_in[3 * i + 2];
                }
            }
            float P[kQ];
            int cur_r = -1;
            warp_by_components<KM, OP>(qtab, K, act, i, x0, x1, x2, ok ? r : -1, a0, a1, a2, P, cur_r,
                                       nullptr, nullptr, nullptr, dir_out, pdf_out, valid_out, sorted_out, base);
            continue;
        }
        // one or two regions for the warp (queries sorted by region; a warp
        // may straddle a region boundary): one pass per region
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            // this pass's region: its records into shared memory
            const int rp = pass == 0 ? r0 : r1;
            if (pass == 1 && r1 == r0) break;
            if (rp != staged) {
                // the region's records, rescaled for the base-2 exponents of
                // both passes: A^-1 and D^-1 times c = sqrt(log2(e) / 2), so that
                // |z|^2 and |y|^2 are already those exponents; C^T times 1 / c
                // (the conditional mean C^T z unchanged); cn times log2(e); cx
                // times log2(e) less the region bound B = log2(e) max_k cx_k:
                // no conditioned weight of the region exceeds 2^B (times the
                // common constant), so 2^(lw - B) needs no per-query maximum
                __syncwarp();
                const float4* src = q4 + (int64_t)rp * n4;
                float cmax = -INFINITY;
                for (int e = lane; e < n4; e += 32) {
                    const int m = e % Q4;
                    float4 v = __ldg(src + e);
                    const float4 f = s_scale[m];
                    cmax = m == 0 ? fmaxf(cmax, v.w) : cmax;
                    v.x *= f.x;
                    v.y *= f.y;
                    v.z *= f.z;
                    v.w *= f.w;
                    s_rec[warp][e] = v;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(FULL, cmax, o));
                const float rbound = cmax > -INFINITY ? cmax * kL2e : 0.f;
                __syncwarp();
                for (int c = lane; c < K; c += 32) {     // cx - B of component c
                    float* cx = &s_rec[warp][c * Q4].w;
                    *cx = fmaf(*cx, kL2e, -rbound);
                }
                __syncwarp();
                staged = rp;
            }
            if (!in || rr != rp) continue;
            const float4* rec = &s_rec[warp][0];

            // ---- pass 1: conditioning on the position (Sec. 3.2), every component:
            // w'_k = 2^(lw - B) with lw = log2 of pi'_k up to a common constant,
            // m = C^T z, se = sum w'_k
            float se = 0.f;
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                // the record's conditioning group as staged, float4 0-4: (mu_x, cx - B),
                // (remainder, c A^-1 0), c A^-1 1..4, (c A^-1 5, C^T row 0 / c),
                // (C^T row 1 / c, 0)
                const float4* rk = rec + k * Q4;
                const float4 g0 = rk[0], g1 = rk[1], g2 = rk[2], g3 = rk[3], g4 = rk[4];
                const float e0 = (x0 - g0.x) - g1.x, e1 = (x1 - g0.y) - g1.y, e2 = (x2 - g0.z) - g1.z;
                const float z0 = g1.w * e0;
                const float z1 = g2.x * e0 + g2.y * e1;
                const float z2 = g2.z * e0 + g2.w * e1 + g3.x * e2;
                const float w = tc::ex2_approx(fmaf(-z2, z2, fmaf(-z1, z1, fmaf(-z0, z0, g0.w))));
                cw[k * CS] = w;
                cmu[k * CS] = make_float2(g3.y * z0 + g3.z * z1 + g3.w * z2, g4.x * z0 + g4.y * z1 + g4.z * z2);
                se += w;
            }
            if (!(se >= 0x1p-100f)) {
                // every weight more than 2^100 below the bound (a position far
                // from all components), where the shifted weights lose
                // precision or flush to zero: w'_k = 2^(lw - max) instead
                float mx = -INFINITY;
#pragma unroll 1
                for (int k = 0; k < K; ++k) {
                    const float4* rk = rec + k * Q4;
                    const float4 g0 = rk[0], g1 = rk[1], g2 = rk[2], g3 = rk[3];
                    const float e0 = (x0 - g0.x) - g1.x, e1 = (x1 - g0.y) - g1.y, e2 = (x2 - g0.z) - g1.z;
                    const float z0 = g1.w * e0;
                    const float z1 = g2.x * e0 + g2.y * e1;
                    const float z2 = g2.z * e0 + g2.w * e1 + g3.x * e2;
                    const float lw = fmaf(-z2, z2, fmaf(-z1, z1, fmaf(-z0, z0, g0.w)));
                    cw[k * CS] = lw;
                    mx = fmaxf(mx, lw);
                }
                se = 0.f;
#pragma unroll 1
                for (int k = 0; k < K; ++k) {
                    const float w = mx > -INFINITY ? tc::ex2_approx(cw[k * CS] - mx) : 0.f;
                    cw[k * CS] = w;
                    se += w;
                }
            }

            float w0, w1, w2;
            int valid = 1;
            if (OP == OP_SAMPLE) {
                float u0, u1, u2;
                if (uni != nullptr) {
                    u0 = uni[3 * i];
                    u1 = uni[3 * i + 1];
                    u2 = uni[3 * i + 2];
                } else {
                    const uint4 o = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 0u),
                                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
                    u0 = u24(o.x);
                    u1 = u24(o.y);
                    u2 = u24(o.z);
                }
                // component by inverse CDF on u0 (Sec. 3.1 "Sampling", step i): the
                // first k with u0 se < cumsum, i.e. the number of partial sums
                // <= u0 se (they do not decrease); rounding past the end takes the
                // last component of positive weight
                const float thr = u0 * se;
                float cum = 0.f;
                int kk = 0;
#pragma unroll 4
                for (int k = 0; k < K; ++k) {
                    cum += cw[k * CS];
                    kk += cum <= thr ? 1 : 0;
                }
                if (kk >= K) {
                    kk = K - 1;
                    while (kk > 0 && !(cw[kk * CS] > 0.f)) --kk;
                }
                const float2 sel = cmu[kk * CS];
                // Gaussian draw in the chart (step ii), exp map (step iii)
                // the chart group, float4 5-8: (t, b.x), (b.y, b.z, mu_w.x, mu_w.y),
                // (mu_w.z, D^-1), (cn, D)
                const float4* rk = rec + kk * Q4;
                const float4 h5 = rk[5], h6 = rk[6], h7 = rk[7], h8 = rk[8];
                const float rad = sqrtf(-2.f * logf(1.f - u1));
                float sn, cs;
                sincospif(2.f * u2, &sn, &cs);
                const float g0 = rad * cs, g1 = rad * sn;
                const float n0 = sel.x + h8.y * g0;
                const float n1 = sel.y + h8.z * g0 + h8.w * g1;
                const float rn = sqrtf(n0 * n0 + n1 * n1);
                valid = (rn < kPiF) && ok && se > 0.f;
                float sr, cr;
                sincosf(rn, &sr, &cr);
                const float sc = rn < 1e-3f ? 1.f - rn * rn * (1.f / 6.f) : __fdividef(sr, rn);
                const float c0 = n0 * sc, c1 = n1 * sc;
                w0 = c0 * h5.x + c1 * h5.w + cr * h6.z;
                w1 = c0 * h5.y + c1 * h6.x + cr * h6.w;
                w2 = c0 * h5.z + c1 * h6.y + cr * h7.x;
            } else {
                w0 = dir_in[3 * i];
                w1 = dir_in[3 * i + 1];
                w2 = dir_in[3 * i + 2];
            }

            // ---- pass 2: solid-angle pdf of the conditioned mixture at w
            // (Sec. 3.1 Eq. solidangle-pdf): sum_k pi'_k N_2(log_k w; m_k, D D^T) / sinc
            float p = 0.f;
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                const float4* rk = rec + k * Q4;
                const float4 h5 = rk[5], h6 = rk[6], h7 = rk[7], h8 = rk[8];   // the chart group
                const float wk = cw[k * CS];
                const float2 mk = cmu[k * CS];
                // t = (h5.x, h5.y, h5.z), b = (h5.w, h6.x, h6.y), mu = (h6.z, h6.w, h7.x)
                const float u = h5.x * w0 + h5.y * w1 + h5.z * w2;
                const float v = h5.w * w0 + h6.x * w1 + h6.y * w2;
                const float cz = h6.z * w0 + h6.w * w1 + h7.x * w2;
                const float s2v = u * u + v * v;
                // antipode of the mean (and within 1e-19 of it): outside the chart
                const bool cut = !(s2v >= 1.17549435e-38f) && cz < 0.f;
                const float gg = cut ? 1.f : g_of_cos(cz, tc::rsqrt_approx(s2v));
                const float d0 = gg * u - mk.x, d1 = gg * v - mk.y;
                // c D^-1 (h7.y, h7.z, h7.w), log2(e) cn = h8.x as staged
                const float y0 = h7.y * d0;
                const float y1 = h7.z * d0 + h7.w * d1;
                const float pk_ = wk * tc::ex2_approx(fmaf(-y1, y1, fmaf(-y0, y0, h8.x))) * gg;
                p += cut ? 0.f : pk_;
            }
            p = se > 0.f ? __fdividef(p, se) : 0.f;
            if (sorted_out != nullptr) {             // the slot's record (binned queries), coalesced
                sorted_out[j] = OP == OP_SAMPLE ? make_float4(w0, w1, w2, valid ? p : -1.f)
                                                : make_float4(ok ? p : 0.f, 0.f, 0.f, 0.f);
            } else if (OP == OP_SAMPLE) {
                dir_out[3 * i] = w0;
                dir_out[3 * i + 1] = w1;
                dir_out[3 * i + 2] = w2;
                valid_out[i] = (uint8_t)valid;
                pdf_out[i] = valid ? p : 0.f;
            } else {
                pdf_out[i] = ok ? p : 0.f;
            }
        }
    }
}

// The queries held by the lanes of one warp (lane l: query il with position
// x, region rr (-1: none) and uniforms or direction a; the lanes in `active`
// hold a query), processed
// SPI = 32/KP at a time with one lane per component; the query's inputs are
// broadcast by shuffles and the component's query record P stays in
// registers while consecutive queries share a region (cur_r).
template <int KP, int OP>
__device__ __forceinline__ void warp_by_components(const float* __restrict__ qtab, int K, unsigned active, int64_t il,
                                                   float x0, float x1, float x2, int rr, float a0, float a1,
                                                   float a2, float* P, int& cur_r, float* __restrict__ cond_pi,
                                                   float* __restrict__ cond_m, float* __restrict__ cond_L,
                                                   float* __restrict__ dir_out, float* __restrict__ pdf_out,
                                                   uint8_t* __restrict__ valid_out, float4* __restrict__ sorted_out,
                                                   int64_t slot0) {
    constexpr int SPI = 32 / KP;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int k = lane & (KP - 1), h = lane / KP, base_lane = h * KP;
    const int n = 32 - __clz(active);           // slots up to the last active lane
    for (int t = 0; t < n; t += SPI) {
        const int j = t + h;
        const bool act = j < 32 && ((active >> j) & 1u);
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
                P[qrec::MUW + 2] = 1.f;
                P[qrec::D] = P[qrec::D + 2] = P[qrec::DINV] = P[qrec::DINV + 2] = 1.f;
                P[qrec::CX] = -INFINITY;
            }
        }
        // ---- conditioning on position: z = A^-1 (x - mu^x)
        const float e0 = (qx0 - P[qrec::MUX]) - P[qrec::REM], e1 = (qx1 - P[qrec::MUX + 1]) - P[qrec::REM + 1],
                    e2 = (qx2 - P[qrec::MUX + 2]) - P[qrec::REM + 2];
        const float z0 = P[qrec::AINV] * e0;
        const float z1 = P[qrec::AINV + 1] * e0 + P[qrec::AINV + 2] * e1;
        const float z2 = P[qrec::AINV + 3] * e0 + P[qrec::AINV + 4] * e1 + P[qrec::AINV + 5] * e2;
        const float lw = P[qrec::CX] - 0.5f * (z0 * z0 + z1 * z1 + z2 * z2);
        const float m0 = P[qrec::CT] * z0 + P[qrec::CT + 1] * z1 + P[qrec::CT + 2] * z2;   // C^T z
        const float m1 = P[qrec::CT + 3] * z0 + P[qrec::CT + 4] * z1 + P[qrec::CT + 5] * z2;
        // normalise pi'_k over the KP component lanes (log-sum-exp)
        float mx = lw;
#pragma unroll
        for (int o = KP / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
        const float e = (mx == -INFINITY) ? 0.f : __expf(lw - mx);
        float se = e;
#pragma unroll
        for (int o = KP / 2; o > 0; o >>= 1) se += __shfl_xor_sync(FULL, se, o);
        const float cpi = se > 0.f ? __fdividef(e, se) : 0.f;
        const int64_t qi = __shfl_sync(FULL, (long long)il, src);

        if (OP == OP_CONDITION) {
            if (act && k < K) {
                const int64_t o = qi * K + k;
                cond_pi[o] = ok ? cpi : 0.f;
                cond_m[2 * o] = m0;
                cond_m[2 * o + 1] = m1;
                cond_L[3 * o] = P[qrec::D];
                cond_L[3 * o + 1] = P[qrec::D + 1];
                cond_L[3 * o + 2] = P[qrec::D + 2];
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
                const float n0 = m0 + P[qrec::D] * g0;
                const float n1 = m1 + P[qrec::D + 1] * g0 + P[qrec::D + 2] * g1;
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
            w1 = __shfl_sync(FULL, s1, from);
            w2 = __shfl_sync(FULL, s2, from);
            valid = __shfl_sync(FULL, vv, from) > 0.5f && ok && pos != 0u;
        }
        // ---- solid-angle pdf of the conditioned mixture at w (Eq. solidangle-pdf)
        const float u = P[qrec::T] * w0 + P[qrec::T + 1] * w1 + P[qrec::T + 2] * w2;
        const float v = P[qrec::B] * w0 + P[qrec::B + 1] * w1 + P[qrec::B + 2] * w2;
        const float cz = P[qrec::MUW] * w0 + P[qrec::MUW + 1] * w1 + P[qrec::MUW + 2] * w2;
        const float s2v = u * u + v * v;
        const bool cut = s2v == 0.f && cz < 0.f;          // antipode: outside the chart
        const float gg = cut ? 1.f : g_of_cos(cz, rsqrtf(s2v));   // theta / sin(theta) = 1/sinc
        const float d0 = gg * u - m0, d1 = gg * v - m1;
        const float y0 = P[qrec::DINV] * d0;
        const float y1 = P[qrec::DINV + 1] * d0 + P[qrec::DINV + 2] * d1;
        float pk_ = cpi * __expf(P[qrec::CN] - 0.5f * (y0 * y0 + y1 * y1)) * gg;
        if (cut || k >= K) pk_ = 0.f;
        float p = pk_;
#pragma unroll
        for (int o = KP / 2; o > 0; o >>= 1) p += __shfl_xor_sync(FULL, p, o);
        if (act && k == 0) {
            if (sorted_out != nullptr) {         // the slot's record (binned queries)
                sorted_out[slot0 + j] = OP == OP_SAMPLE ? make_float4(w0, w1, w2, valid ? p : -1.f)
                                                        : make_float4(ok ? p : 0.f, 0.f, 0.f, 0.f);
            } else if (OP == OP_SAMPLE) {
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

template <int KP, int OP>
__global__ void __launch_bounds__(256)
    k_query(const float* __restrict__ qtab, int K, int64_t R, int64_t Q,
            const float* __restrict__ qx, const int32_t* __restrict__ region, GridF grid,
            uint64_t seed, const float* __restrict__ uni, const float* __restrict__ dir_in,
            float* __restrict__ cond_pi, float* __restrict__ cond_m, float* __restrict__ cond_L,
            float* __restrict__ dir_out, float* __restrict__ pdf_out,
            uint8_t* __restrict__ valid_out) {
    const int lane = threadIdx.x & 31;
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
        warp_by_components<KP, OP>(qtab, K, __ballot_sync(0xffffffffu, i < Q), i, x0, x1, x2, rr, a0, a1, a2, P,
                                   cur_r, cond_pi, cond_m, cond_L, dir_out, pdf_out, valid_out, nullptr, 0);
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

// ---------------------------------------------------------------------------
// Binning of queries given in any order: a counting sort by region.
//   k_qbin_keys     region of every query (array or grid; out of range: bin R)
//                   and the per-bin counts (warp-aggregated atomics)
//   k_qbin_scan     exclusive prefix sum of the R + 1 counts, each rounded up
//                   to a multiple of 32 (one CTA, 8 counts per thread and
//                   round), so that every bin starts
//                   at a multiple of 32 and no warp of the sampling kernel
//                   spans two regions
//   k_qbin_scatter  each query's position (slot) in its bin (warp-aggregated
//                   atomic cursor): perm[slot] = query index and inv[query] =
//                   slot; the padding slots keep perm = -1 (no query)
//   k_qbin_unpermute  the sampling kernel writes each slot's outputs as one
//                   16-byte record in slot order (coalesced); query i then
//                   gathers its record from slot inv[i] and writes its outputs
//                   in query order, so no output is written at random
// The order within a bin depends on the atomics; no result does, since every
// query's output depends only on its own inputs and index.
__global__ void __launch_bounds__(256) k_qbin_keys(int64_t Q, int64_t R, const float* __restrict__ qx,
                                                   const int32_t* __restrict__ region, GridF grid,
                                                   int32_t* __restrict__ key, int32_t* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < Q; base += wstride) {
        const int64_t i = base + lane;
        int r = -1;
        if (i < Q) {
            if (region != nullptr) {
                r = region[i];
            } else {
                const float xs[3] = {qx[3 * i], qx[3 * i + 1], qx[3 * i + 2]};
                int id[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int v = (int)floorf((xs[c] - grid.lo[c]) * grid.scale[c]);
                    id[c] = min(max(v, 0), grid.dims[c] - 1);
                }
                r = id[0] + grid.dims[0] * (id[1] + grid.dims[1] * id[2]);
            }
            if (r < 0 || r >= R) r = (int)R;
            key[i] = r;
        }
        const unsigned m = __match_any_sync(0xffffffffu, r);
        if (i < Q && lane == __ffs(m) - 1) atomicAdd(counts + r, __popc(m));
    }
}

__global__ void __launch_bounds__(1024) k_qbin_scan(int64_t n, int32_t* __restrict__ v) {
    // each thread takes 8 consecutive counts per round (8,192 per round, so
    // 65,537 bins in nine rounds of one block-wide scan)
    constexpr int PER = 8;
    __shared__ int32_t s_warp[32];
    __shared__ int32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024 * PER) {
        const int64_t e0 = base + (int64_t)tid * PER;
        int32_t c[PER];
        int32_t x = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            c[q] = e0 + q < n ? (v[e0 + q] + 31) & ~31 : 0;   // bin sizes padded to whole warps
            x += c[q];
        }
        const int32_t own = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += u;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t w = s_warp[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int32_t incl = x + (warp > 0 ? s_warp[warp - 1] : 0);
        int32_t run = s_carry + incl - own;                   // exclusive prefix of this thread's first count
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (e0 + q < n) v[e0 + q] = run;
            run += c[q];
        }
        __syncthreads();
        if (tid == 1023) s_carry += incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_qbin_scatter(int64_t Q, const int32_t* __restrict__ key_in,
                                                      int32_t* __restrict__ cursor, int32_t* __restrict__ perm,
                                                      int32_t* __restrict__ inv) {
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < Q; base += wstride) {
        const int64_t i = base + lane;
        const int r = i < Q ? key_in[i] : -1;
        const unsigned m = __match_any_sync(0xffffffffu, r);
        const int leader = __ffs(m) - 1;
        int32_t pos = 0;
        if (i < Q && lane == leader) pos = atomicAdd(cursor + r, __popc(m));
        pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(m & ((1u << lane) - 1u));
        if (i < Q) {
            perm[pos] = (int32_t)i;
            inv[i] = pos;
        }
    }
}

// The slots' records back to the queries' own indices: query i reads its
// slot inv[i] (a 16-byte gather) and writes its outputs in order.
template <int OP>
__global__ void __launch_bounds__(256) k_qbin_unpermute(int64_t Q, const int32_t* __restrict__ inv,
                                                        const float4* __restrict__ rec, float* __restrict__ dir_out,
                                                        float* __restrict__ pdf_out, uint8_t* __restrict__ valid_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += stride) {
        const float4 v = rec[inv[i]];
        if (OP == OP_SAMPLE) {
            dir_out[3 * i] = v.x;
            dir_out[3 * i + 1] = v.y;
            dir_out[3 * i + 2] = v.z;
            pdf_out[i] = fmaxf(v.w, 0.f);
            valid_out[i] = (uint8_t)(v.w >= 0.f);
        } else {
            pdf_out[i] = v.x;
        }
    }
}

// sorted positions, padding included: Q + 31 per bin at most
static int64_t qbin_slots(int64_t R, int64_t Q) { return Q + 31 * (R + 1); }

size_t qbin_workspace_bytes(int64_t R, int64_t Q) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(sizeof(int32_t) * (size_t)(R + 1)) + 2 * up(sizeof(int32_t) * (size_t)Q) +
           up(sizeof(int32_t) * (size_t)qbin_slots(R, Q)) + up(sizeof(float4) * (size_t)qbin_slots(R, Q));
}

cudaError_t launch_query_binned(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K, int64_t R,
                                int64_t Q, const float* qx, const int32_t* region, const GridF& g, uint64_t seed,
                                const float* uni, const float* dir_in, float* dir_out, float* pdf_out,
                                uint8_t* valid_out, void* ws) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t slots = qbin_slots(R, Q);
    unsigned char* p = static_cast<unsigned char*>(ws);
    int32_t* counts = reinterpret_cast<int32_t*>(p);
    p += up(sizeof(int32_t) * (size_t)(R + 1));
    int32_t* key = reinterpret_cast<int32_t*>(p);
    p += up(sizeof(int32_t) * (size_t)Q);
    int32_t* inv = reinterpret_cast<int32_t*>(p);
    p += up(sizeof(int32_t) * (size_t)Q);
    int32_t* perm = reinterpret_cast<int32_t*>(p);
    p += up(sizeof(int32_t) * (size_t)slots);
    float4* rec = reinterpret_cast<float4*>(p);
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)(R + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(perm, 0xff, sizeof(int32_t) * (size_t)slots, s);   // -1: padding
    if (e != cudaSuccess) return e;
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((Q + 255) / 256, (int64_t)grid * 4));
    k_qbin_keys<<<gb, 256, 0, s>>>(Q, R, qx, region, g, key, counts);
    k_qbin_scan<<<1, 1024, 0, s>>>(R + 1, counts);
    k_qbin_scatter<<<gb, 256, 0, s>>>(Q, key, counts, perm, inv);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_query_q(s, op, KP, grid, qtab, K, R, slots, qx, region, g, perm, rec, seed, uni, dir_in, dir_out,
                       pdf_out, valid_out);
    if (e != cudaSuccess) return e;
    if (op == OP_SAMPLE)
        k_qbin_unpermute<OP_SAMPLE><<<gb, 256, 0, s>>>(Q, inv, rec, dir_out, pdf_out, valid_out);
    else
        k_qbin_unpermute<OP_PDF><<<gb, 256, 0, s>>>(Q, inv, rec, dir_out, pdf_out, valid_out);
    return cudaGetLastError();
}

cudaError_t launch_query_q(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K, int64_t R,
                           int64_t Q, const float* qx, const int32_t* region, const GridF& g, const int32_t* perm,
                           float4* sorted_out, uint64_t seed, const float* uni, const float* dir_in,
                           float* dir_out, float* pdf_out, uint8_t* valid_out) {
    // a persistent grid: every resident CTA walks the queries with a stride
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    (void)grid;
    const int64_t blocks = (Q + kQWarps * 32 - 1) / (kQWarps * 32);
    const int gq = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)nsm * kQCtas));
#define SDMM_QQ(M)                                                                                           \
    case M:                                                                                                  \
        if (op == OP_SAMPLE)                                                                                 \
            k_query_q<M, OP_SAMPLE><<<gq, kQWarps * 32, 0, s>>>(qtab, K, R, Q, qx, region, g, perm, sorted_out, seed, \
                                                                uni, dir_in, dir_out, pdf_out, valid_out);   \
        else                                                                                                 \
            k_query_q<M, OP_PDF><<<gq, kQWarps * 32, 0, s>>>(qtab, K, R, Q, qx, region, g, perm, sorted_out, seed,    \
                                                             uni, dir_in, dir_out, pdf_out, valid_out);      \
        break;
    switch (KP) {
        SDMM_QQ(1)
        SDMM_QQ(2)
        SDMM_QQ(4)
        SDMM_QQ(8)
        SDMM_QQ(16)
        default: return cudaErrorInvalidValue;
    }
#undef SDMM_QQ
    return cudaGetLastError();
}

cudaError_t launch_query(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K,
                         int64_t R, int64_t Q, const float* qx, const int32_t* region,
                         const GridF& g, uint64_t seed, const float* uni, const float* dir_in,
                         float* cond_pi, float* cond_m, float* cond_L, float* dir_out,
                         float* pdf_out, uint8_t* valid_out) {
    // sampling and pdf with up to 16 components: one thread per query
    if (op != OP_CONDITION && KP <= 16)
        return launch_query_q(s, op, KP, grid, qtab, K, R, Q, qx, region, g, nullptr, nullptr, seed, uni, dir_in,
                              dir_out, pdf_out, valid_out);
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
