// estep.cu -- E-step + statistics of the plain fit on the CUDA cores (sm_103a):
// the tangent-space (chart) density of Sec. 3.2 Eq. (em-ss-computation) with
// the log map of Sec. 3.1 Eq. (log), one lane per mixture component.
//
// This is the specialisation of k_accumulate<KP, MODE_FIT> for the chart
// density and tangent charts (the default configuration and the batched fit's
// whole E-step).  It computes the same quantities with less work per
// (sample, component) pair:
//   * base 2 throughout: L^-1 is scaled by sqrt(log2(e) / 2) when a region's
//     records are loaded, so the Mahalanobis sum of squares is already the
//     base-2 exponent, and the per-component constant c5 is stored shifted by
//     the region bound (the largest c5 of the region, which no component's
//     chart density can exceed), so exp(l - bound) is one ex2;
//   * positions relative to a per-unit reference point (the region's first
//     spatial mean, FP32): the sample's offset is formed once per sample when
//     it is staged, each component's mean offset once per region, so the pair
//     needs one subtraction per coordinate, with no hi/lo correction;
//   * the statistics are taken in the whitened chart coordinates
//     y = sqrt(log2(e) / 2) L^-1 d, which the Mahalanobis term computes
//     anyway: y = L'^-1 (x', g u, g v) - b with b = L'^-1 (mean offsets) per
//     component, so no d is formed; the M-step takes them back to the chart
//     (s1 = L s1_y / c, s2 = L s2_y L^T / c^2, FP64);
//   * two samples per lane in flight (samples t + h and t + SPI + h), so the
//     two log-sum-exp butterflies and the two MUFU chains overlap;
//   * the next batch of 32 samples is loaded while the current one is processed.
// Samples whose shifted sum underflows (every component more than ~69 below
// the region bound) get no statistics in the pass and are redone after their
// batch with the exact per-sample maximum, as in k_accumulate.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace sdmm {

namespace {
constexpr int kEW = 4;                          // warps per CTA
constexpr int kECtas = 5;                       // resident CTAs per SM (96 registers per thread)
constexpr float kLog2eF = 1.44269504088896341f;
constexpr float kLn2F = 0.693147180559945309f;
constexpr float kHalfLog2eSqrt = 0.849321800288019f;   // sqrt(log2(e) / 2)
constexpr float kSumMin = 1e-30f;               // smallest trusted shifted sum

// *p = (a, b) in shared memory if `pred`, as one predicated store
__device__ __forceinline__ void st_shared_pred(bool pred, float2* p, float a, float b) {
    const uint32_t addr = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.v2.f32 [%1], {%2, %3};\n\t}" ::"r"((int)pred),
        "r"(addr), "f"(a), "f"(b)
        : "memory");
}
}  // namespace

// OFFS: records carry an in-chart direction offset (the objective at offset
// means, and the Euclidean ablation's mean); EUCL: the Euclidean ablation
// (direction coordinates without the log map, g = 1); SOLID: the solid-angle
// density p^t / sinc of the E-step, whose log Jacobian lifts a component above
// the region bound, so every sample takes the exact per-sample maximum.
// TWO: the second pass of the accurate covariance update (Sec. 3.2 Eq.
// tangent-space-sigma-update): the responsibilities of the current
// parameters, the sample measured in the chart of each component's new mean
// (chart2 records: new mean, its rows t', b', mu'), and only the second
// moments w r d' d'^T accumulated, 15 per component, in the chart.
template <int KP, bool OFFS, bool EUCL, bool SOLID, bool TWO = false>
__global__ void __launch_bounds__(kEW * 32, kECtas)
    k_estep(WsHeader* __restrict__ ws, const int64_t* __restrict__ chunk_base,
            const int32_t* __restrict__ chunk_region, const float* __restrict__ etab, int K, int chunk,
            float* __restrict__ partial, int ps, int write_ll, const float* __restrict__ chart2) {
    static_assert(!(TWO && (OFFS || EUCL)), "the second pass runs in tangent charts at the means");
    static_assert(KP >= 4 && KP <= 32, "two samples per lane need 2 * 32 / KP <= 32");
    constexpr int SPI = 32 / KP;
    constexpr int RED = KP * kStat + 4;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ __align__(16) float4 s_x[kEW][32];   // (x - xref, weight) of the batch's samples
    __shared__ __align__(16) float4 s_w[kEW][32];   // (direction, 0)
    __shared__ float2 s_lse[kEW][32];               // per sample: (shifted sum, shift)
    __shared__ float red[kEW][RED];
    __shared__ int s_c;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = lane & (KP - 1), h = lane / KP;
    const float* __restrict__ px = ws->desc.p[0];
    const float* __restrict__ py = ws->desc.p[1];
    const float* __restrict__ pz = ws->desc.p[2];
    const float* __restrict__ ox = ws->desc.p[3];
    const float* __restrict__ oy = ws->desc.p[4];
    const float* __restrict__ oz = ws->desc.p[5];
    const float* __restrict__ pw = ws->desc.p[6];
    const int64_t* __restrict__ off = ws->desc.offsets;
    float* __restrict__ loglik = write_ll ? ws->desc.loglik : nullptr;
    const int n_chunks = ws->n_chunks;
    const int64_t R = ws->desc.R;

    // this lane's component: R_mu rows (t, b, mu), mo = the scaled L^-1 times
    // the mean's offset from the reference point and, with OFFS (the
    // objective at offset means, the Euclidean mean), the in-chart direction
    // offset; li = the scaled L^-1; base-2 constant shifted by the region bound
    float rt[9], mo[5], li[15];
#pragma unroll
    for (int q = 0; q < 9; ++q) rt[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 5; ++q) mo[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 15; ++q) li[q] = 0.f;
    float c2 = -INFINITY, lmax = 0.f;
    float xr0 = 0.f, xr1 = 0.f, xr2 = 0.f;
    float n2[9] = {}, mo2[3] = {};   // TWO: the new chart's rows and mean (from the reference point); unused otherwise
    int prev_r = -1;

    // log2 of the chart density of one sample at this lane's component,
    // relative to the region bound; y receives the whitened tangent vector
    auto logp2 = [&](const float4 sa, const float4 sb, float y[5]) -> float {
        const float u = rt[0] * sb.x + rt[1] * sb.y + rt[2] * sb.z;
        const float v = rt[3] * sb.x + rt[4] * sb.y + rt[5] * sb.z;
        const float cz = rt[6] * sb.x + rt[7] * sb.y + rt[8] * sb.z;
        const float s2 = u * u + v * v;
        // 1/sin(theta) clamped so that g stays finite (and d with it) at the
        // antipode of the mean, which has no chart: its density is 0 below
        const float gg = EUCL ? 1.f : g_of_cos_fit(cz, fminf(tc::rsqrt_approx(s2), 1e18f));
        const float gu = gg * u, gv = gg * v;
        y[0] = fmaf(li[0], sa.x, -mo[0]);
        y[1] = fmaf(li[2], sa.y, fmaf(li[1], sa.x, -mo[1]));
        y[2] = fmaf(li[5], sa.z, fmaf(li[4], sa.y, fmaf(li[3], sa.x, -mo[2])));
        y[3] = fmaf(li[9], gu, fmaf(li[8], sa.z, fmaf(li[7], sa.y, fmaf(li[6], sa.x, -mo[3]))));
        y[4] = fmaf(li[14], gv, fmaf(li[13], gu, fmaf(li[12], sa.z, fmaf(li[11], sa.y,
                                                                           fmaf(li[10], sa.x, -mo[4])))));
        float l2 = fmaf(-y[0], y[0], c2);
        l2 = fmaf(-y[1], y[1], l2);
        l2 = fmaf(-y[2], y[2], l2);
        l2 = fmaf(-y[3], y[3], l2);
        l2 = fmaf(-y[4], y[4], l2);
        if (SOLID) l2 += tc::lg2_approx(gg);                       // p^t / sinc: + log2(theta / sin)
        if (EUCL) return l2;
        const bool cut = !(s2 >= 1.17549435e-38f) && cz < 0.f;   // to within 1e-19 rad
        return cut ? -INFINITY : l2;
    };

    // TWO: the sample in the chart of this lane's component's new mean,
    // d' = (x - mu'^x, log_{mu'}(w)), into y; true at the new chart's cut locus
    auto new_chart = [&](const float4 sa, const float4 sb, float y[5]) -> bool {
        const float u = n2[0] * sb.x + n2[1] * sb.y + n2[2] * sb.z;
        const float v = n2[3] * sb.x + n2[4] * sb.y + n2[5] * sb.z;
        const float cz = n2[6] * sb.x + n2[7] * sb.y + n2[8] * sb.z;
        const float s2 = u * u + v * v;
        const float gg = g_of_cos_fit(cz, fminf(tc::rsqrt_approx(s2), 1e18f));
        y[0] = sa.x - mo2[0];
        y[1] = sa.y - mo2[1];
        y[2] = sa.z - mo2[2];
        y[3] = gg * u;
        y[4] = gg * v;
        return !(s2 >= 1.17549435e-38f) && cz < 0.f;
    };

    for (;;) {
        if (threadIdx.x == 0) s_c = atomicAdd(&ws->queue, 1);
        __syncthreads();
        const int c = s_c;
        if (c >= n_chunks) break;
        const int r = chunk_region[c];
        if (r < 0 || r >= R) {               // never happens for units built by k_build_chunks
            __syncthreads();                 // (uniform branch) s_c is read before it is rewritten
            continue;
        }
        const int64_t o1 = off[r + 1];
        const int64_t start = off[r] + ((int64_t)c - chunk_base[r]) * chunk;
        const int64_t end = min(start + (int64_t)chunk, o1);
        if (r != prev_r) {
            prev_r = r;
            const float* rec0 = etab + (int64_t)r * K * kE;
            xr0 = __ldg(rec0 + 0);
            xr1 = __ldg(rec0 + 1);
            xr2 = __ldg(rec0 + 2);
            float c5 = -INFINITY;
            if (k < K) {
                float p[kE];
                const float4* src = reinterpret_cast<const float4*>(rec0 + (int64_t)k * kE);
#pragma unroll
                for (int q = 0; q < kE / 4; ++q) {
                    const float4 v = __ldg(src + q);
                    p[4 * q + 0] = v.x;
                    p[4 * q + 1] = v.y;
                    p[4 * q + 2] = v.z;
                    p[4 * q + 3] = v.w;
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) rt[q] = p[3 + q];
#pragma unroll
                for (int q = 0; q < 15; ++q) li[q] = p[12 + q] * kHalfLog2eSqrt;
                // the mean relative to the reference point, whitened
                const float m[5] = {(p[0] - xr0) + p[32], (p[1] - xr1) + p[33], (p[2] - xr2) + p[34],
                                    OFFS ? p[28] : 0.f, OFFS ? p[29] : 0.f};
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    float acc_m = 0.f;
#pragma unroll
                    for (int b = 0; b <= a; ++b) acc_m = fmaf(li[pk(a, b)], m[b], acc_m);
                    mo[a] = acc_m;
                }
                c5 = p[27];
                if (TWO) {
                    float q2[kChart];
                    const float4* src2 = reinterpret_cast<const float4*>(chart2 + ((int64_t)r * K + k) * kChart);
#pragma unroll
                    for (int q = 0; q < kChart / 4; ++q) {
                        const float4 v = __ldg(src2 + q);
                        q2[4 * q + 0] = v.x;
                        q2[4 * q + 1] = v.y;
                        q2[4 * q + 2] = v.z;
                        q2[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int q = 0; q < 9; ++q) n2[q] = q2[3 + q];
#pragma unroll
                    for (int c = 0; c < 3; ++c) mo2[c] = ((c == 0 ? q2[0] : c == 1 ? q2[1] : q2[2]) -
                                                          (c == 0 ? xr0 : c == 1 ? xr1 : xr2)) + q2[12 + c];
                }
            } else {                         // padding lane: density 0
#pragma unroll
                for (int q = 0; q < 9; ++q) rt[q] = 0.f;
                rt[8] = 1.f;
#pragma unroll
                for (int q = 0; q < 5; ++q) mo[q] = 0.f;
#pragma unroll
                for (int q = 0; q < 15; ++q) li[q] = 0.f;
                if (TWO) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) n2[q] = 0.f;
                    n2[8] = 1.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) mo2[q] = 0.f;
                }
            }
            lmax = c5;
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(FULL, lmax, o));
            if (!(lmax > -INFINITY)) lmax = 0.f;      // every weight zero: all densities are 0
            c2 = (c5 - lmax) * kLog2eF;               // -inf for zero weights and padding lanes
        }

        // the statistics [s0, s1 (5), s2 (15, packed)]; five pairs of them sit
        // in float2 registers for the packed FP32 instructions of sm_100+
        // (one instruction, two lanes' worth of FMA): s1 (0, 1) and (2, 3),
        // s2 (0,0)+(1,1), (2,2)+(3,3) and (2,0)+(3,1)
        float a_s0 = 0.f, a_s14 = 0.f, a_10 = 0.f, a_21 = 0.f, a_30 = 0.f, a_32 = 0.f;
        float a_4[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        float2 a_s101 = make_float2(0.f, 0.f), a_s123 = make_float2(0.f, 0.f);
        float2 a_d01 = make_float2(0.f, 0.f), a_d23 = make_float2(0.f, 0.f), a_x = make_float2(0.f, 0.f);
        float wsum = 0.f, wll = 0.f;

        // statistics [1, y, y y^T] of one pair, weighted by w r: the products
        // w_a y_b (w_a = w r y_a, a >= b) of the scalar form, 20 instructions
        auto accumulate = [&](const float wr, const float y[5]) {
            const float2 y01 = make_float2(y[0], y[1]), y23 = make_float2(y[2], y[3]);
            const float2 wr2 = make_float2(wr, wr);
            const float2 w01 = __fmul2_rn(wr2, y01), w23 = __fmul2_rn(wr2, y23);
            const float w4 = wr * y[4];
            a_s0 += wr;
            a_s101 = __fadd2_rn(a_s101, w01);
            a_s123 = __fadd2_rn(a_s123, w23);
            a_s14 += w4;
            a_d01 = __ffma2_rn(w01, y01, a_d01);
            a_d23 = __ffma2_rn(w23, y23, a_d23);
            a_x = __ffma2_rn(w23, y01, a_x);
            a_10 = fmaf(w01.y, y[0], a_10);
            a_21 = fmaf(w23.x, y[1], a_21);
            a_30 = fmaf(w23.y, y[0], a_30);
            a_32 = fmaf(w23.y, y[2], a_32);
#pragma unroll
            for (int b = 0; b < 5; ++b) a_4[b] = fmaf(w4, y[b], a_4[b]);
        };

        // raw values of this lane's sample of the next batch
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, f4 = 0.f, f5 = 1.f, f6 = 0.f;
        auto fetch = [&](const int64_t i) {
            if (i < end) {
                f0 = __ldg(px + i);
                f1 = __ldg(py + i);
                f2 = __ldg(pz + i);
                f3 = __ldg(ox + i);
                f4 = __ldg(oy + i);
                f5 = __ldg(oz + i);
                f6 = __ldg(pw + i);
            } else {
                f0 = f1 = f2 = f3 = f4 = f6 = 0.f;
                f5 = 1.f;
            }
        };
        fetch(start + warp * 32 + lane);

        for (int64_t g = start + warp * 32; g < end; g += kEW * 32) {
            // stage this batch (past the unit: weight 0, a valid direction)
            const float my_w = f6;
            s_x[warp][lane] = make_float4(f0 - xr0, f1 - xr1, f2 - xr2, f6);
            s_w[warp][lane] = make_float4(f3, f4, f5, 0.f);
            __syncwarp();
            fetch(g + kEW * 32 + lane);
            const int n = (int)min((int64_t)32, end - g);

            for (int t = 0; t < n; t += 2 * SPI) {
                const int ja = t + h, jb = t + SPI + h;   // both < 32; past n they carry weight 0
                const float4 xa = s_x[warp][ja], wa = s_w[warp][ja];
                const float4 xb = s_x[warp][jb], wb = s_w[warp][jb];
                float ya[5], yb[5];
                const float la = logp2(xa, wa, ya), lb = logp2(xb, wb, yb);
                float refa = 0.f, refb = 0.f;       // shift on top of the region bound
                if (SOLID) {                         // the two maxima, reduce-scatter as the sums below
                    const bool up = (k & (KP / 2)) != 0;
                    float keep = up ? lb : la;
                    keep = fmaxf(keep, __shfl_xor_sync(FULL, up ? la : lb, KP / 2));
#pragma unroll
                    for (int o = KP / 4; o > 0; o >>= 1) keep = fmaxf(keep, __shfl_xor_sync(FULL, keep, o));
                    const float other = __shfl_xor_sync(FULL, keep, KP / 2);
                    refa = up ? other : keep;
                    refb = up ? keep : other;
                    refa = refa == -INFINITY ? 0.f : refa;
                    refb = refb == -INFINITY ? 0.f : refb;
                }
                const float ea = tc::ex2_approx(la - refa);
                const float eb = tc::ex2_approx(lb - refb);
                // the two sums by one reduce-scatter: at the first level the lower
                // half of the sample's lanes keeps sample a, the upper half b; each
                // half then reduces one value; a last exchange returns both
                // (five shuffles instead of eight)
                float sa, sb;
                {
                    const bool up = (k & (KP / 2)) != 0;
                    float keep = up ? eb : ea;
                    keep += __shfl_xor_sync(FULL, up ? ea : eb, KP / 2);
#pragma unroll
                    for (int o = KP / 4; o > 0; o >>= 1) keep += __shfl_xor_sync(FULL, keep, o);
                    const float other = __shfl_xor_sync(FULL, keep, KP / 2);
                    sa = up ? other : keep;
                    sb = up ? keep : other;
                }
                // component lane 0 records sample a's sum, lane KP/2 sample b's (one
                // predicated store: no branch in the pair loop)
                {
                    const bool lo = k == 0;
                    st_shared_pred(lo || k == KP / 2, &s_lse[warp][lo ? ja : jb], lo ? sa : sb,
                                   SOLID ? lmax + (lo ? refa : refb) * kLn2F : lmax);
                }
                const float ia = tc::rcp_approx(sa), ib = tc::rcp_approx(sb);
                float ra = sa >= kSumMin ? xa.w * ea * ia : 0.f;
                float rb = sb >= kSumMin ? xb.w * eb * ib : 0.f;
                if (TWO) {
                    if (new_chart(xa, wa, ya)) ra = 0.f;
                    if (new_chart(xb, wb, yb)) rb = 0.f;
                }
                accumulate(ra, ya);
                accumulate(rb, yb);
            }
            __syncwarp();
            // samples whose shifted sum underflowed: again with the exact maximum
            unsigned redo = __ballot_sync(FULL, lane < n && !(s_lse[warp][lane].x >= kSumMin));
            while (redo) {
                // slot h takes the (h+1)-th lowest flagged sample (none: 0xffffffff)
                const unsigned jj = __fns(redo, 0u, h + 1);
#pragma unroll
                for (int hh = 0; hh < SPI; ++hh) redo &= redo - 1u;
                const bool act = jj < 32u;
                const int j = act ? (int)jj : 0;
                const float4 xa = s_x[warp][j], wa = s_w[warp][j];
                float ya[5];
                const float l2 = logp2(xa, wa, ya);
                float ref = l2;
#pragma unroll
                for (int o = KP / 2; o > 0; o >>= 1) ref = fmaxf(ref, __shfl_xor_sync(FULL, ref, o));
                const float e = (ref == -INFINITY) ? 0.f : tc::ex2_approx(l2 - ref);
                float se = e;
#pragma unroll
                for (int o = KP / 2; o > 0; o >>= 1) se += __shfl_xor_sync(FULL, se, o);
                if (k == 0 && act) s_lse[warp][j] = make_float2(se, lmax + ref * kLn2F);
                float rr = (act && se >= kSumMin) ? __fdividef(xa.w * e, se) : 0.f;
                if (TWO && new_chart(xa, wa, ya)) rr = 0.f;
                accumulate(rr, ya);
            }
            __syncwarp();
            // lane i: log-likelihood, weight and weighted log-likelihood of sample g + i
            {
                const float2 q = s_lse[warp][lane];
                if (lane < n) {
                    const float li_ = (q.x > 0.f) ? q.y + __logf(q.x) : -INFINITY;
                    wsum += my_w;
                    wll += (my_w > 0.f) ? my_w * li_ : 0.f;
                    if (loglik != nullptr) loglik[g + lane] = li_;
                }
            }
            __syncwarp();
        }
        // back to [s0, s1, s2 packed]
        float acc[kStat];
        acc[0] = a_s0;
        acc[1] = a_s101.x, acc[2] = a_s101.y, acc[3] = a_s123.x, acc[4] = a_s123.y, acc[5] = a_s14;
        acc[6 + pk(0, 0)] = a_d01.x, acc[6 + pk(1, 1)] = a_d01.y;
        acc[6 + pk(2, 2)] = a_d23.x, acc[6 + pk(3, 3)] = a_d23.y;
        acc[6 + pk(2, 0)] = a_x.x, acc[6 + pk(3, 1)] = a_x.y;
        acc[6 + pk(1, 0)] = a_10, acc[6 + pk(2, 1)] = a_21, acc[6 + pk(3, 0)] = a_30, acc[6 + pk(3, 2)] = a_32;
#pragma unroll
        for (int b = 0; b < 5; ++b) acc[6 + pk(4, b)] = a_4[b];
        // combine the SPI sample slots of each component; W and sum w l over all lanes
#pragma unroll
        for (int o = KP; o < 32; o <<= 1) {
#pragma unroll
            for (int s = 0; s < kStat; ++s) acc[s] += __shfl_xor_sync(FULL, acc[s], o);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wsum += __shfl_xor_sync(FULL, wsum, o);
            wll += __shfl_xor_sync(FULL, wll, o);
        }
        if (h == 0 && k < K) {
#pragma unroll
            for (int s = 0; s < kStat; ++s) red[warp][k * kStat + s] = acc[s];
        }
        if (lane == 0) {
            red[warp][K * kStat] = wsum;
            red[warp][K * kStat + 1] = wll;
        }
        __syncthreads();
        if (TWO) {   // the second pass's layout: 15 second moments per component
            const int nv = K * 15;
            for (int v = threadIdx.x; v < nv; v += kEW * 32) {
                const int src = (v / 15) * kStat + 6 + v % 15;
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < kEW; ++w) s += red[w][src];
                partial[(int64_t)c * ps + v] = s;
            }
        } else {
            const int nv = K * kStat + 2;
            for (int v = threadIdx.x; v < nv; v += kEW * 32) {
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < kEW; ++w) s += red[w][v];
                partial[(int64_t)c * ps + v] = s;
            }
        }
    }
}

bool estep_fast_supported(int KP) { return KP >= 4 && KP <= 32; }

cudaError_t launch_estep_fast(cudaStream_t s, int KP, int grid, WsHeader* ws, const int64_t* cb,
                              const int32_t* cr, const float* etab, int K, int chunk, float* partial,
                              int ps, int write_ll, int variant, const float* chart2) {
    // persistent grid of every resident CTA (the work queue balances the
    // units); the caller's grid, sized for the 8-warp kernels, is not used
    (void)grid;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid = nsm * kECtas;
#define SDMM_ESTEP_V(P, O, E, S, T)                                                                    \
    k_estep<P, O, E, S, T><<<grid, kEW * 32, 0, s>>>(ws, cb, cr, etab, K, chunk, partial, ps, write_ll, chart2)
#define SDMM_ESTEP(P)                                                                                  \
    case P:                                                                                            \
        if (variant == ESTEP_EUCLID) SDMM_ESTEP_V(P, true, true, false, false);                        \
        else if (variant == ESTEP_SOLID) SDMM_ESTEP_V(P, false, false, true, false);                   \
        else if (variant == ESTEP_SOLID_OFFSETS) SDMM_ESTEP_V(P, true, false, true, false);            \
        else if (variant == ESTEP_OFFSETS) SDMM_ESTEP_V(P, true, false, false, false);                 \
        else if (variant == ESTEP_TWO) SDMM_ESTEP_V(P, false, false, false, true);                     \
        else if (variant == ESTEP_TWO_SOLID) SDMM_ESTEP_V(P, false, false, true, true);                \
        else SDMM_ESTEP_V(P, false, false, false, false);                                              \
        break;
    switch (KP) {
        SDMM_ESTEP(4)
        SDMM_ESTEP(8)
        SDMM_ESTEP(16)
        SDMM_ESTEP(32)
        default: return cudaErrorInvalidValue;
    }
#undef SDMM_ESTEP
#undef SDMM_ESTEP_V
    return cudaGetLastError();
}

}  // namespace sdmm
