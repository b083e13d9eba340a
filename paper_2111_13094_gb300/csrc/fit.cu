// fit.cu -- SDMM fitting kernels for sm_103a.
//
//  k_set_desc       writes the batch descriptor into the workspace
//  k_build_chunks   splits every region into work units of `chunk` samples
//  k_accumulate     persistent E-step + statistics (or adjoint statistics):
//                   one lane per mixture component, FP32, per-unit partials
//  k_reduce_mstep   FP64 fixed-order reduction of a region's partials, then
//                   Robbins-Monro averaging and the MAP M-step
//  k_reduce_objective  MAP objective and its adjoint from the partials
//  k_init_regions   initialisation (k-means++ seeds, App. B covariances)
//  k_prepare        derived FP32 records from the FP64 parameters
#include "common.cuh"
#include "kernels.h"

namespace sdmm {

__global__ void k_set_desc(WsHeader* ws, BatchDesc d) { ws->desc = d; }

// ---------------------------------------------------------------------------
// Work units.  Region r with M_r >= min_samples samples gets ceil(M_r/chunk)
// units; chunk_base is the exclusive prefix sum over regions (int64 scan),
// chunk_region the owner of each unit.  Units beyond the workspace capacity
// `max_chunks` (possible only when offsets overlap) are not created; the
// M-step flags their regions.  When `units` is given, it receives each unit's
// sample range [start, end) (the tensor-core E-step reads it).  One CTA of
// 1024 threads.
__global__ void __launch_bounds__(1024) k_build_chunks(WsHeader* ws, int64_t* chunk_base,
                                                       int32_t* chunk_region, int64_t* units, int chunk,
                                                       int min_samples, int64_t max_chunks) {
    const int64_t R = ws->desc.R, N = ws->desc.N;
    const int64_t* off = ws->desc.offsets;
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < R; base += 1024) {
        const int64_t r = base + tid;
        int64_t n = 0;
        if (r < R) {
            const int64_t o0 = off[r], o1 = off[r + 1];
            const bool ok = o0 >= 0 && o1 >= o0 && o1 <= N;
            const int64_t M = o1 - o0;
            if (ok && M >= min_samples && M > 0) n = (M + chunk - 1) / chunk;
        }
        int64_t v = n;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = s_warp[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int64_t incl = v + (warp > 0 ? s_warp[warp - 1] : 0);
        if (r < R) chunk_base[r] = s_carry + incl - n;
        __syncthreads();
        if (tid == 1023) s_carry += incl;
        __syncthreads();
    }
    const int64_t total = s_carry;
    if (tid == 0) {
        chunk_base[R] = total;
        ws->n_chunks = (int32_t)min(total, max_chunks);
        ws->queue = 0;
        ws->err = 0;
    }
    __syncthreads();   // chunk_base is complete before any thread reads a neighbour's entry
    for (int64_t r = tid; r < R; r += 1024) {
        const int64_t c0 = chunk_base[r];
        const int64_t c1 = min(r + 1 < R ? chunk_base[r + 1] : total, max_chunks);
        for (int64_t c = c0; c < c1; ++c) {
            chunk_region[c] = (int32_t)r;
            if (units != nullptr) {               // sample range [start, end) of unit c
                const int64_t start = off[r] + (c - c0) * chunk;
                units[2 * c] = start;
                units[2 * c + 1] = min(start + (int64_t)chunk, off[r + 1]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// E-step + statistics.  A CTA of 8 warps takes work units from a global queue.
// Within a warp, lane = (h, k): k = lane % KP is the mixture component and
// h = lane / KP selects one of SPI = 32/KP samples processed side by side, so
// each lane keeps its component's parameters and its 21 accumulators in
// registers for the whole unit.  Samples are read coalesced (one per lane per
// stream) into a per-warp shared buffer and then broadcast to the KP lanes of
// each sample.  The per-sample log-sum-exp over components is a butterfly
// over the KP lanes.
//
// MODE_FIT  accumulates w r [1, d, d d^T]          (Sec. 3.2 Eq. em-ss-computation)
// MODE_GRAD accumulates w r [1, z, z y^T], y = L^-1 d, z = L^-T y (adjoint)
// Both also accumulate W = sum w and sum w l_i.
// MODE_TWO  (second pass of the accurate covariance update, Sec. 3.2
//           Eq. tangent-space-sigma-update) keeps the responsibilities of the
//           current parameters but measures d' = (x - mu'^x, log_{mu'}(w)) in
//           the chart of each component's new mean mu' (chart2 records) and
//           accumulates only w r d' d'^T.
constexpr int kWarps = 8;
// A sum of exp(l - region bound) below kLseMin means every component lies more
// than ~69 below the bound, near the bottom of the FP32 range where the
// exponentials are flushed or held at the smallest normal: the sum then says
// nothing about the sample, and the exact per-sample maximum is used instead.
constexpr float kLseMin = 1e-30f;

template <int KP, int MODE>
__global__ void __launch_bounds__(kWarps * 32, 2)
    k_accumulate(WsHeader* __restrict__ ws, const int64_t* __restrict__ chunk_base,
                 const int32_t* __restrict__ chunk_region, const float* __restrict__ etab, int K,
                 int chunk, int density, float* __restrict__ partial, int ps, int write_ll,
                 const float* __restrict__ chart2, int euclid) {
    constexpr int SPI = 32 / KP;
    constexpr int NS = MODE == MODE_TWO ? 15 : kStat;   // statistics per component
    constexpr int RED = KP * kStat + 4;
    __shared__ __align__(16) float sbuf[kWarps][32][8];
    __shared__ float2 s_lse[kWarps][32];   // per sample of the batch: (sum of exp, shift)
    __shared__ float red[kWarps][RED];
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

    float prm[kE];
    float c2[MODE == MODE_TWO ? kChart : 1];
    float lmax = 0.f;
    int prev_r = -1;
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
            if (k < K) {
                const float4* src = reinterpret_cast<const float4*>(etab + ((int64_t)r * K + k) * kE);
#pragma unroll
                for (int q = 0; q < kE / 4; ++q) {
                    const float4 v = __ldg(src + q);
                    prm[4 * q + 0] = v.x;
                    prm[4 * q + 1] = v.y;
                    prm[4 * q + 2] = v.z;
                    prm[4 * q + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kE; ++q) prm[q] = 0.f;
                prm[11] = 1.f;
                prm[27] = -INFINITY;
            }
            if (MODE == MODE_TWO) {
                if (k < K) {
                    const float4* src = reinterpret_cast<const float4*>(chart2 + ((int64_t)r * K + k) * kChart);
#pragma unroll
                    for (int q = 0; q < kChart / 4; ++q) {
                        const float4 v = __ldg(src + q);
                        c2[4 * q + 0] = v.x;
                        c2[4 * q + 1] = v.y;
                        c2[4 * q + 2] = v.z;
                        c2[4 * q + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kChart; ++q) c2[q] = 0.f;
                    c2[11] = 1.f;
                }
            }
            // upper bound of every component's log-density in this region:
            // l_k = c5_k - q/2 <= c5_k (tangent density), so exp(l - lmax) <= 1
            lmax = prm[27];
#pragma unroll
            for (int o = KP / 2; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        }
        float acc[kStat];
#pragma unroll
        for (int s = 0; s < kStat; ++s) acc[s] = 0.f;
        float wsum = 0.f, wll = 0.f;

        for (int64_t g = start + warp * 32; g < end; g += kWarps * 32) {
            const int64_t i = g + lane;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 1.f, 0.f);
            if (i < end) {
                a = make_float4(__ldg(px + i), __ldg(py + i), __ldg(pz + i), __ldg(pw + i));
                b = make_float4(__ldg(ox + i), __ldg(oy + i), __ldg(oz + i), 0.f);
            }
            *reinterpret_cast<float4*>(&sbuf[warp][lane][0]) = a;
            *reinterpret_cast<float4*>(&sbuf[warp][lane][4]) = b;
            const float my_w = a.w;                 // weight of sample g + lane (0 past the unit)
            __syncwarp();
            const int n = (int)min((int64_t)32, end - g);
            // one (sample j, this lane's component) pair: log-likelihood, the
            // sample's log-sum-exp over the component lanes, statistics.
            // lse: 0 = shift by the region bound, the exact maximum when that
            // underflows (a warp vote); 1 = the bound only (an underflowing
            // sample gets no statistics and is redone after the batch);
            // 2 = the exact maximum.  act = false: weight 0 (idle slot).
            auto pair = [&](const int j, const bool act, const int lse) {
                const float4 sa = *reinterpret_cast<const float4*>(&sbuf[warp][j][0]);
                const float4 sb = *reinterpret_cast<const float4*>(&sbuf[warp][j][4]);
                // log map at this lane's component (Sec. 3.1 Eq. log); the
                // Euclidean ablation has unit rows and no change of variables
                const float u = prm[3] * sb.x + prm[4] * sb.y + prm[5] * sb.z;
                const float v = prm[6] * sb.x + prm[7] * sb.y + prm[8] * sb.z;
                float gg = 1.f;
                bool cut = false;
                if (!euclid) {
                    const float cz = prm[9] * sb.x + prm[10] * sb.y + prm[11] * sb.z;
                    const float s2 = u * u + v * v;
                    cut = s2 == 0.f && cz < 0.f;     // cut locus: undefined chart
                    gg = cut ? 1.f : g_of_cos(cz, rsqrtf(s2));
                }
                float d[5];
                d[0] = (sa.x - prm[0]) - prm[32];
                d[1] = (sa.y - prm[1]) - prm[33];
                d[2] = (sa.z - prm[2]) - prm[34];
                d[3] = gg * u - prm[28];
                d[4] = gg * v - prm[29];
                const float* Li = prm + 12;
                float y[5];
                y[0] = Li[0] * d[0];
                y[1] = Li[1] * d[0] + Li[2] * d[1];
                y[2] = Li[3] * d[0] + Li[4] * d[1] + Li[5] * d[2];
                y[3] = Li[6] * d[0] + Li[7] * d[1] + Li[8] * d[2] + Li[9] * d[3];
                y[4] = Li[10] * d[0] + Li[11] * d[1] + Li[12] * d[2] + Li[13] * d[3] + Li[14] * d[4];
                const float q = y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3] + y[4] * y[4];
                float l = prm[27] - 0.5f * q;
                if (density) l += __logf(gg);
                if (cut) l = -INFINITY;
                // log-sum-exp over the KP component lanes of this sample
                float ref = lmax, e = 0.f, se = 0.f;
                if (lse != 2) {
                    e = __expf(l - ref);
                    se = e;
#pragma unroll
                    for (int o = KP / 2; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
                }
                if (lse == 2 || (lse == 0 && __any_sync(0xffffffffu, !(se >= kLseMin) || se > 1e30f || density))) {
                    ref = l;
#pragma unroll
                    for (int o = KP / 2; o > 0; o >>= 1) ref = fmaxf(ref, __shfl_xor_sync(0xffffffffu, ref, o));
                    e = (ref == -INFINITY) ? 0.f : __expf(l - ref);
                    se = e;
#pragma unroll
                    for (int o = KP / 2; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
                }
                const float rr = (se >= kLseMin) ? __fdividef(e, se) : 0.f;
                const float wt = act ? sa.w : 0.f;
                const float wr = wt * rr;
                // the sample's log-likelihood is formed once per batch, below
                if (MODE != MODE_TWO && k == 0 && act) s_lse[warp][j] = make_float2(se, ref);
                if (MODE == MODE_TWO) {
                    // the sample in the chart of the new mean: same log map, new centre
                    const float u2 = c2[3] * sb.x + c2[4] * sb.y + c2[5] * sb.z;
                    const float v2 = c2[6] * sb.x + c2[7] * sb.y + c2[8] * sb.z;
                    const float cz2 = c2[9] * sb.x + c2[10] * sb.y + c2[11] * sb.z;
                    const float s22 = u2 * u2 + v2 * v2;
                    const bool cut2 = s22 == 0.f && cz2 < 0.f;   // cut locus of the new chart
                    const float g2 = cut2 ? 1.f : g_of_cos(cz2, rsqrtf(s22));
                    float dn[5];
                    dn[0] = (sa.x - c2[0]) - c2[12];
                    dn[1] = (sa.y - c2[1]) - c2[13];
                    dn[2] = (sa.z - c2[2]) - c2[14];
                    dn[3] = g2 * u2;
                    dn[4] = g2 * v2;
                    const float wr2 = cut2 ? 0.f : wr;
#pragma unroll
                    for (int a2 = 0; a2 < 5; ++a2) {
                        const float wa = wr2 * dn[a2];
#pragma unroll
                        for (int b2 = 0; b2 <= a2; ++b2) acc[pk(a2, b2)] += wa * dn[b2];
                    }
                    return;
                }
                float x[5];
                if (MODE == MODE_FIT) {
#pragma unroll
                    for (int a2 = 0; a2 < 5; ++a2) x[a2] = d[a2];
                } else {
                    x[4] = Li[14] * y[4];
                    x[3] = Li[9] * y[3] + Li[13] * y[4];
                    x[2] = Li[5] * y[2] + Li[8] * y[3] + Li[12] * y[4];
                    x[1] = Li[2] * y[1] + Li[4] * y[2] + Li[7] * y[3] + Li[11] * y[4];
                    x[0] = Li[0] * y[0] + Li[1] * y[1] + Li[3] * y[2] + Li[6] * y[3] + Li[10] * y[4];
#pragma unroll
                    for (int a2 = 0; a2 < 5; ++a2) d[a2] = y[a2];
                }
                acc[0] += wr;
#pragma unroll
                for (int a2 = 0; a2 < 5; ++a2) {
                    const float wa = wr * x[a2];
                    acc[1 + a2] += wa;
#pragma unroll
                    for (int b2 = 0; b2 <= a2; ++b2) acc[6 + pk(a2, b2)] += wa * d[b2];
                }
            };
            // the plain fit defers underflowing samples (rare: every component
            // below the region bound by more than ~87 in log) instead of
            // voting on every sample
            const bool defer = MODE == MODE_FIT && !density;
#pragma unroll 2
            for (int t = 0; t < n; t += SPI) pair(t + h, true, defer ? 1 : 0);
            if (defer) {
                __syncwarp();
                unsigned redo = __ballot_sync(0xffffffffu, lane < n && !(s_lse[warp][lane].x >= kLseMin));
                while (redo) {
                    // slot h takes the h-th lowest flagged sample
                    unsigned m = redo;
                    int jj = -1;
                    for (int hh = 0; hh <= h && m; ++hh) {
                        jj = __ffs(m) - 1;
                        m &= m - 1u;
                        if (hh < h && !m) jj = -1;
                    }
                    for (int hh = 0; hh < SPI && redo; ++hh) redo &= redo - 1u;
                    pair(jj >= 0 ? jj : 0, jj >= 0, 2);
                }
            }
            __syncwarp();
            if (MODE != MODE_TWO) {
                // lane i: log-likelihood, weight and weighted log-likelihood of sample g + i
                const float2 q = s_lse[warp][lane];
                if (lane < n) {
                    const float li = (q.x > 0.f) ? q.y + __logf(q.x) : -INFINITY;
                    wsum += my_w;
                    wll += (my_w > 0.f) ? my_w * li : 0.f;
                    if (loglik != nullptr) loglik[g + lane] = li;
                }
                __syncwarp();
            }
        }
        // combine the SPI sample slots of each component; W and sum w l over all lanes
#pragma unroll
        for (int o = KP; o < 32; o <<= 1) {
#pragma unroll
            for (int s = 0; s < NS; ++s) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], o);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
            wll += __shfl_xor_sync(0xffffffffu, wll, o);
        }
        if (h == 0 && k < K) {
#pragma unroll
            for (int s = 0; s < NS; ++s) red[warp][k * NS + s] = acc[s];
        }
        if (MODE != MODE_TWO && lane == 0) {
            red[warp][K * NS] = wsum;
            red[warp][K * NS + 1] = wll;
        }
        __syncthreads();
        const int nv = K * NS + (MODE == MODE_TWO ? 0 : 2);
        for (int v = threadIdx.x; v < nv; v += kWarps * 32) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += red[w][v];
            partial[(int64_t)c * ps + v] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Sum of a region's unit partials in FP64, in unit order (deterministic).
// The units' FP32 partials of one region summed in a fixed order: four
// consecutive units in FP32 (pairwise), the groups in FP64.  FP64 work on
// GB300's narrow FP64 pipe is what bounds the M-step; a unit partial carries
// the rounding of its own FP32 accumulation over up to thousands of samples,
// which the three FP32 additions of a group do not exceed.
__device__ inline void reduce_partials(const float* __restrict__ partial, int ps, int64_t c0,
                                       int64_t c1, int nv, double* __restrict__ out, int t0 = threadIdx.x,
                                       int nt = blockDim.x) {
    for (int v = t0; v < nv; v += nt) {
        const float* __restrict__ p = partial + v;
        double s = 0.0;
        int64_t c = c0;
        for (; c + 4 <= c1; c += 4)
            s += (double)((p[c * ps] + p[(c + 1) * ps]) + (p[(c + 2) * ps] + p[(c + 3) * ps]));
        for (; c < c1; ++c) s += (double)p[c * ps];
        out[v] = s;
    }
}

// Statistics of the specialised E-step (k_estep) come in the whitened chart
// coordinates y = c L^-1 d of each component (c = sqrt(log2(e) / 2), the
// FP32 constant of that kernel): back to the chart, s1 = L s1_y / c and
// s2 = L s2_y L^T / c^2 (sk = [s0, s1 (5), s2 (15, packed)], FP64).
__device__ inline void whitened_to_chart(const double* __restrict__ L, double* __restrict__ sk) {
    const double c = (double)0.849321800288019f;
    const double ic = 1.0 / c, ic2 = ic * ic;      // folded at compile time: no FP64 division per entry
    double Y[5][5], T[5][5];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b <= a; ++b) Y[a][b] = Y[b][a] = sk[6 + pk(a, b)];
    double s1[5];
    for (int i = 0; i < 5; ++i) {
        double v = 0.0;
        for (int j = 0; j <= i; ++j) v += L[pk(i, j)] * sk[1 + j];
        s1[i] = v * ic;
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double v = 0.0;
            for (int m = 0; m <= i; ++m) v += L[pk(i, m)] * Y[m][j];
            T[i][j] = v;
        }
    for (int i = 0; i < 5; ++i) {
        sk[1 + i] = s1[i];
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int m = 0; m <= j; ++m) v += T[i][m] * L[pk(j, m)];
            sk[6 + pk(i, j)] = v * ic2;
        }
    }
}

__device__ inline double prior_beta(const sdmm_config& cfg, const double* prior_scale,
                                    int64_t r, int64_t seen) {
    if (cfg.prior_scale_mode == SDMM_PRIOR_SCALE_ARRAY && prior_scale != nullptr)
        return prior_scale[r];
    return seen > 0 ? 1.0 / (double)seen : 0.0;
}

// ---------------------------------------------------------------------------
// FP64 reduction + averaging + MAP M-step, one CTA per region (Sec. 3.2,
// Sec. 3.4, Sec. 4.3).  Thread k < K updates component k.
// Feature-space statistics of one component (contraction form) to the
// chart statistics [s0, s1 (5), s2 (15)].  Rows a, b, c hold sums of
// w r phi, w r g phi and w r g^2 phi over the features
// phi = [1, x', vech(x'x'), w, w (x) x', vech(ww)] with x' = x - xref.
//
// Euclidean ablation: g = 1 (the three rows agree), unit rows A = (e_x, e_y)
// and the direction measured from the mean, nu = A w - (mu_x, mu_y): the
// statistics of nu pick up the offset terms below.
__device__ inline void features_to_stats(const double* Fa, const double* Fb, const double* Fc,
                                         const double mp[3], const double muw[3], double* out,
                                         bool euclid = false) {
    double t[3], b[3];
    if (euclid) {
        t[0] = 1.0, t[1] = 0.0, t[2] = 0.0;
        b[0] = 0.0, b[1] = 1.0, b[2] = 0.0;
    } else {
        basis_f64(muw, t, b);
    }
    const double A[2][3] = {{t[0], t[1], t[2]}, {b[0], b[1], b[2]}};
    static constexpr int V[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};   // vech index of (p, q)
    const double s0 = Fa[0];
    const double Sx[3] = {Fa[1], Fa[2], Fa[3]};
    double* s1 = out + 1;
    double* s2 = out + 6;
    out[0] = s0;
    for (int a = 0; a < 3; ++a) s1[a] = Sx[a] - mp[a] * s0;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c <= a; ++c)
            s2[pk(a, c)] = Fa[4 + V[a][c]] - mp[a] * Sx[c] - Sx[a] * mp[c] + s0 * mp[a] * mp[c];
    const double Gw[3] = {Fb[10], Fb[11], Fb[12]};
    for (int j = 0; j < 2; ++j) {
        s1[3 + j] = A[j][0] * Gw[0] + A[j][1] * Gw[1] + A[j][2] * Gw[2];
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            for (int p = 0; p < 3; ++p) v += A[j][p] * (Fb[13 + 3 * p + a] - mp[a] * Gw[p]);
            s2[pk(3 + j, a)] = v;
        }
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) v += A[i][p] * Fc[22 + V[p][q]] * A[j][q];
            s2[pk(3 + i, 3 + j)] = v;
        }
    if (euclid) {
        // sums of A w are in s1[3..4] and s2[(3+i), *]; shift them by o = (mu_x, mu_y)
        const double o[2] = {muw[0], muw[1]};
        const double aw[2] = {s1[3], s1[4]};
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j <= i; ++j)
                s2[pk(3 + i, 3 + j)] += -o[i] * aw[j] - aw[i] * o[j] + s0 * o[i] * o[j];
        for (int i = 0; i < 2; ++i) {
            for (int a = 0; a < 3; ++a) s2[pk(3 + i, a)] -= o[i] * s1[a];
            s1[3 + i] = aw[i] - o[i] * s0;
        }
    }
}

// Second-pass charts of the accurate covariance update: per component the
// batch mean offset m = s1 / s0 of the first pass (FP64 sums of the unit
// partials), the new mean (mu^x + m^x, exp_{mu^w}(m^nu), Eq. tangent-space-
// mu-update) and its chart rows, as kChart floats: mu^x hi, t, b, mu^w,
// mu^x lo.  Also re-arms the work queue for the second pass.
__global__ void __launch_bounds__(128) k_new_charts(WsHeader* __restrict__ ws,
                                                    const int64_t* __restrict__ chunk_base,
                                                    const float* __restrict__ partial, int ps,
                                                    sdmm_config cfg, sdmm_state st,
                                                    float* __restrict__ chart2, int ystats) {
    const int64_t r = blockIdx.x;
    const int K = cfg.K;
    const int tid = threadIdx.x;
    __shared__ double s_st[SDMM_MAX_K * kStat];
    if (r == 0 && tid == 0) ws->queue = 0;
    const int64_t nc = ws->n_chunks;
    reduce_partials(partial, ps, min(chunk_base[r], nc), min(chunk_base[r + 1], nc), K * kStat, s_st);
    __syncthreads();
    if (tid < K) {
        const int64_t rk = r * K + tid;
        if (ystats) whitened_to_chart(st.L + rk * 15, s_st + tid * kStat);
        const double s0 = s_st[tid * kStat];
        double m[5], nmx[3], omw[3], nmw[3], t[3], b[3];
        for (int c = 0; c < 5; ++c) m[c] = (s0 > 0.0 && isfinite(s0)) ? s_st[tid * kStat + 1 + c] / s0 : 0.0;
        for (int c = 0; c < 3; ++c) {
            nmx[c] = st.mu_x[rk * 3 + c] + m[c];
            omw[c] = st.mu_w[rk * 3 + c];
        }
        exp_map_f64(omw, m + 3, nmw);
        basis_f64(nmw, t, b);
        float* o = chart2 + rk * kChart;
        for (int c = 0; c < 3; ++c) {
            const float hi = (float)nmx[c];
            o[c] = hi;
            o[12 + c] = (float)(nmx[c] - (double)hi);
            o[3 + c] = (float)t[c];
            o[6 + c] = (float)b[c];
            o[9 + c] = (float)nmw[c];
        }
        o[15] = 0.f;
    }
}


// G regions per CTA: with one-warp CTAs and K <= 16, lanes 0-15 update the
// components of one region and lanes 16-31 those of the next.  A warp's FP64
// instruction occupies the SM's FP64 pipe equally long with 16 or 32 active
// lanes, and this kernel is bound by that pipe, so two regions per warp halve
// its time.  Threads of a group: gsz = blockDim.x / G; thread k < K of the
// group updates component k; the group's threads share the reduction.  The
// packed form is capped at 128 registers so that 16 one-warp CTAs fit on an
// SM and the 4,096-region fit's 2,048 CTAs run in one wave (a few spilled
// FP64 values cost less than a second, nearly empty wave).
template <bool FEAT, bool TWO, int G>
__global__ void __launch_bounds__(G == 1 ? 128 : 32, G == 1 ? 1 : 16) k_reduce_mstep(WsHeader* __restrict__ ws,
                                                      const int64_t* __restrict__ chunk_base,
                                                      const float* __restrict__ partial, int ps,
                                                      sdmm_config cfg, sdmm_state st, int iter,
                                                      const float* __restrict__ xref,
                                                      const float* __restrict__ partial2, int ps2,
                                                      int ystats, int64_t R) {
    static_assert(G == 1 || (!FEAT && 32 % G == 0), "packed regions: plain statistics, one warp");
    constexpr int KC = G == 1 ? SDMM_MAX_K : 32 / G;      // components per group, at most
    const int K = cfg.K;
    const int gsz = blockDim.x / G;
    const int grp = threadIdx.x / gsz, tid = threadIdx.x - grp * gsz;
    const int64_t r = (int64_t)blockIdx.x * G + grp;
    const bool have = r < R;
    __shared__ double s_stg[G][KC * kStat + 2];
    __shared__ double s_feat[FEAT ? 3 * SDMM_MAX_K * kFeat + 8 : 1];
    __shared__ double s_S0g[G][KC];
    __shared__ double s_twog[TWO ? G : 1][TWO ? KC * 15 : 1];   // second-pass moments (accurate update)
    __shared__ int s_codeg[G][KC];
    __shared__ int s_skip[G];
    double* const s_st = s_stg[grp];
    double* const s_S0 = s_S0g[grp];
    double* const s_two = s_twog[TWO ? grp : 0];
    int* const s_code = s_codeg[grp];

    // the accumulate kernel of this step has finished: re-arm its work queue
    if (blockIdx.x == 0 && threadIdx.x == 0) ws->queue = 0;
    int64_t o0 = 0, o1 = 0, c0 = 0, c1 = 0;
    if (have) {
        o0 = ws->desc.offsets[r];
        o1 = ws->desc.offsets[r + 1];
        c0 = chunk_base[r];
        c1 = chunk_base[r + 1];
    }
    const int64_t M = o1 - o0;
    const int64_t n_chunks = ws->n_chunks;
    if (tid == 0) {
        int code = -1;  // -1: proceed
        if (!have) {
            code = 0;
        } else if (iter == 0) {
            if (!(o0 >= 0 && o1 >= o0 && o1 <= ws->desc.N) || c1 > n_chunks)
                code = SDMM_REGION_BAD_OFFSETS;
            else if (M < cfg.min_samples || M <= 0) code = SDMM_REGION_SKIPPED;
            if (code >= 0) st.status[r] = code;
        } else if (st.status[r] != SDMM_REGION_OK && st.status[r] != SDMM_REGION_REPAIRED) {
            code = st.status[r];
        }
        s_skip[grp] = code;
    }
    __syncthreads();
    bool alive = s_skip[grp] < 0;
    // (every thread reaches each __syncthreads below; dead groups only skip work)
    if (FEAT) {
        if (alive) reduce_partials(partial, ps, c0, c1, 3 * K * kFeat + 8, s_feat, tid, gsz);
        __syncthreads();
        if (alive && tid < K) {
            const int64_t rk = r * K + tid;
            double mp[3], muw[3];
            for (int c = 0; c < 3; ++c) {
                mp[c] = st.mu_x[rk * 3 + c] - (double)xref[r * 4 + c];
                muw[c] = st.mu_w[rk * 3 + c];
            }
            features_to_stats(s_feat + tid * kFeat, s_feat + (K + tid) * kFeat,
                              s_feat + (2 * K + tid) * kFeat, mp, muw, s_st + tid * kStat,
                              cfg.dir_coords == SDMM_DIR_EUCLIDEAN);
        }
        if (alive && tid == 0) {   // W and sum w l arrive as four per-quadrant parts each
            const double* wq = s_feat + 3 * K * kFeat;
            s_st[K * kStat] = (wq[0] + wq[1]) + (wq[2] + wq[3]);
            s_st[K * kStat + 1] = (wq[4] + wq[5]) + (wq[6] + wq[7]);
        }
    } else {
        if (alive) reduce_partials(partial, ps, c0, c1, K * kStat + 2, s_st, tid, gsz);
        if (ystats) {
            __syncthreads();
            if (alive)
                for (int k = tid; k < K; k += gsz) whitened_to_chart(st.L + (r * K + k) * 15, s_st + k * kStat);
        }
    }
    if (TWO && alive) reduce_partials(partial2, ps2, c0, c1, K * 15, s_two, tid, gsz);
    __syncthreads();
    const double W = alive ? s_st[K * kStat] : 0.0;
    if (tid == 0 && alive) {
        int code = -1;
        if (ws->err != 0) code = SDMM_REGION_DEVICE_TIMEOUT;
        else if (!isfinite(W)) code = SDMM_REGION_NONFINITE;
        else if (!(W > 0.0)) code = SDMM_REGION_ZERO_WEIGHT;
        if (code >= 0) st.status[r] = code;
        s_skip[grp] = code;
    }
    __syncthreads();
    alive = alive && s_skip[grp] < 0;

    int64_t seen = 0;
    double beta = 0.0, eta = 1.0;
    if (alive) {
        seen = (iter == 0) ? st.n_seen[r] + M : st.n_seen[r];
        beta = prior_beta(cfg, ws->desc.prior_scale, r, seen);
        if (cfg.eta_mode != SDMM_ETA_ONE) {
            // (0.1 j + 1)^-alpha; the paper's alpha = 1/2 as one reciprocal square root
            const double base = cfg.eta_beta * (double)st.step_j[r] + 1.0;
            eta = cfg.eta_alpha == 0.5 ? rsqrt(base) : pow(base, -cfg.eta_alpha);
        }
    }
    const double q = cfg.prior_q / K, a = cfg.prior_a / K;
    const bool euclid = cfg.dir_coords == SDMM_DIR_EUCLIDEAN;

    double nmx[3], nmw[3], nL[15], nS2[15], hS0 = 0.0;
    int code = 0;
    const int64_t rk = r * K + tid;
    if (alive && tid < K) {
        const double* sk = s_st + tid * kStat;
        const double invW = 1.0 / W;
        // Robbins-Monro average of the normalised batch statistics; the
        // stored first moment is zero (centred at the current mean)
        hS0 = (1.0 - eta) * st.S0[rk] + eta * (sk[0] * invW);
        double m[5], hS2[15];
        bool fin = isfinite(hS0);
        const double inv0 = hS0 > 0.0 ? 1.0 / hS0 : 0.0;
        for (int c = 0; c < 5; ++c) {
            const double h1 = eta * (sk[1 + c] * invW);
            fin = fin && isfinite(h1);
            m[c] = h1 * inv0;
        }
        for (int p = 0; p < 15; ++p) {
            hS2[p] = (1.0 - eta) * st.S2[rk * 15 + p] + eta * (sk[6 + p] * invW);
            fin = fin && isfinite(hS2[p]);
        }
        if (!fin) {
            code = SDMM_REGION_NONFINITE;
        } else {
            double omx[3], omw[3];
            for (int c = 0; c < 3; ++c) {
                omx[c] = st.mu_x[rk * 3 + c];
                omw[c] = st.mu_w[rk * 3 + c];
                nmx[c] = omx[c] + m[c];
            }
            double J[4] = {1.0, 0.0, 0.0, 1.0};        // chart change (Sec. 3.4), identity if Euclidean
            if (euclid) {                                 // ablation: translate (x, y)
                nmw[0] = omw[0] + m[3];
                nmw[1] = omw[1] + m[4];
                nmw[2] = omw[2];
            } else {
                exp_map_jacobian_f64(omw, m + 3, nmw, J);   // Eq. tangent-space-mu-update
            }
            if (TWO) {
                // accurate update (Eq. tangent-space-sigma-update): the second
                // pass measured the batch in the new chart, centred at the new mean
                for (int p = 0; p < 15; ++p) nS2[p] = s_two[tid * 15 + p] * invW;
            } else {
                // centred second moment in the old chart ...
                double C[15];
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j <= i; ++j) C[pk(i, j)] = hS2[pk(i, j)] - hS0 * m[i] * m[j];
                // ... moved to the new chart: T C T^T, T = blockdiag(I3, J) (Sec. 3.4)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j <= i; ++j) nS2[pk(i, j)] = C[pk(i, j)];
                for (int ia = 0; ia < 2; ++ia)
                    for (int j = 0; j < 3; ++j)
                        nS2[pk(3 + ia, j)] = J[ia * 2 + 0] * C[pk(3, j)] + J[ia * 2 + 1] * C[pk(4, j)];
                const double c33 = C[pk(3, 3)], c43 = C[pk(4, 3)], c44 = C[pk(4, 4)];
                for (int ia = 0; ia < 2; ++ia)
                    for (int ib = 0; ib <= ia; ++ib) {
                        const double a0 = J[ia * 2 + 0], a1 = J[ia * 2 + 1];
                        const double b0 = J[ib * 2 + 0], b1 = J[ib * 2 + 1];
                        nS2[pk(3 + ia, 3 + ib)] =
                            a0 * (c33 * b0 + c43 * b1) + a1 * (c43 * b0 + c44 * b1);
                    }
            }
            // MAP covariance (Sec. 4.3)
            const double Bd[5] = {a * cfg.prior_B_pos, a * cfg.prior_B_pos, a * cfg.prior_B_pos,
                                  a * cfg.prior_B_dir, a * cfg.prior_B_dir};
            const double iden = 1.0 / (beta * a + hS0);
            double Sig[15];
            for (int i = 0; i < 5; ++i)
                for (int j = 0; j <= i; ++j)
                    Sig[pk(i, j)] = ((i == j ? beta * Bd[i] : 0.0) + nS2[pk(i, j)]) * iden;
            if (!cholesky5_f64(Sig, nL)) {
                // numerical floor: smallest tau * B / a (tau = 1e-6 ... 1) that
                // makes the covariance positive definite; the region is flagged
                code = SDMM_REGION_NUMERIC;
                for (double tau = 1e-6; tau <= 1.0; tau *= 100.0) {
                    double Sf[15];
                    for (int p = 0; p < 15; ++p) Sf[p] = Sig[p];
                    for (int c = 0; c < 5; ++c) Sf[pk(c, c)] += tau * Bd[c] / a;
                    if (cholesky5_f64(Sf, nL)) {
                        code = SDMM_REGION_REPAIRED;
                        break;
                    }
                }
            }
        }
        s_code[tid] = code;
        s_S0[tid] = hS0;
    }
    __syncthreads();
    if (alive && tid == 0) {
        int first = 0, repaired = 0;
        for (int kk = 0; kk < K && first == 0; ++kk) {
            if (s_code[kk] == SDMM_REGION_REPAIRED) repaired = 1;
            else first = s_code[kk];
        }
        s_skip[grp] = first;
        if (first != 0) st.status[r] = first;
        s_code[0] = repaired;
    }
    __syncthreads();
    alive = alive && s_skip[grp] == 0;
    if (!alive) return;                      // no barrier follows
    const bool repaired = s_code[0] != 0;
    if (tid < K) {
        double sumS0 = 0.0;
        for (int kk = 0; kk < K; ++kk) sumS0 += s_S0[kk];
        const double npi = (beta * q + hS0) / (K * beta * q + sumS0);  // MAP weights
        st.pi[rk] = npi;
        for (int c = 0; c < 3; ++c) {
            st.mu_x[rk * 3 + c] = nmx[c];
            st.mu_w[rk * 3 + c] = nmw[c];
        }
        for (int p = 0; p < 15; ++p) {
            st.L[rk * 15 + p] = nL[p];
            st.S2[rk * 15 + p] = nS2[p];
        }
        st.S0[rk] = hS0;
        write_records(npi, nmx, nmw, nL, st.etab + rk * kE, st.qtab + rk * kQ, nullptr, euclid);
    }
    if (tid == 0) {
        st.Wbar[r] = (1.0 - eta) * st.Wbar[r] + eta * (W / (double)M);
        st.step_j[r] += 1;
        st.n_seen[r] = seen;
        // a repair in any step of this call is reported (later steps continue)
        if (repaired) st.status[r] = SDMM_REGION_REPAIRED;
        else if (iter == 0) st.status[r] = SDMM_REGION_OK;
    }
}

// ---------------------------------------------------------------------------
// MAP objective (and, with dF != nullptr, its adjoint) from the partials.
// The adjoint's statistics [w r, w r z, w r z y^T (lower)] (z = L^-T y,
// y = L^-1 d) from the whitened ones of the specialised E-step,
// [w r, w r y', w r y' y'^T] with y' = c y (c = sqrt(log2(e) / 2)): z is
// L^-T y per component, so its sums are L^-T times the sums of y.  FP64.
__device__ inline void whitened_to_adjoint(const double* __restrict__ Li, double* __restrict__ sk) {
    const double ic = 1.0 / (double)0.849321800288019f, ic2 = ic * ic;
    double Y[5][5], z1[5], zy[15];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b <= a; ++b) Y[a][b] = Y[b][a] = sk[6 + pk(a, b)];
    for (int i = 0; i < 5; ++i) {
        double v = 0.0;
        for (int m = i; m < 5; ++m) v += Li[pk(m, i)] * sk[1 + m];
        z1[i] = v * ic;
        for (int j = 0; j <= i; ++j) {
            double u = 0.0;
            for (int m = i; m < 5; ++m) u += Li[pk(m, i)] * Y[m][j];
            zy[pk(i, j)] = u * ic2;
        }
    }
    for (int i = 0; i < 5; ++i) sk[1 + i] = z1[i];
    for (int p = 0; p < 15; ++p) sk[6 + p] = zy[p];
}

__global__ void __launch_bounds__(128) k_reduce_objective(
    const WsHeader* __restrict__ ws, const int64_t* __restrict__ chunk_base,
    const float* __restrict__ partial, int ps, sdmm_config cfg, sdmm_state st, double* F_out,
    const double* __restrict__ dF, float* g_delta, float* g_L, float* g_logit, int ystats) {
    const int64_t r = blockIdx.x;
    const int K = cfg.K;
    const int tid = threadIdx.x;
    __shared__ double s_st[SDMM_MAX_K * kStat + 2];
    __shared__ double s_Fk[SDMM_MAX_K];
    const int64_t nc = ws->n_chunks;
    reduce_partials(partial, ps, min(chunk_base[r], nc), min(chunk_base[r + 1], nc), K * kStat + 2, s_st);
    __syncthreads();
    const double W = s_st[K * kStat];
    const double beta = prior_beta(cfg, ws->desc.prior_scale, r, st.n_seen[r]);
    const double q = cfg.prior_q / K, a = cfg.prior_a / K;
    if (tid < K) {
        const int64_t rk = r * K + tid;
        const double* L = st.L + rk * 15;
        double Li[15];
        lower_inverse5_f64(L, Li);
        const double Bd[5] = {a * cfg.prior_B_pos, a * cfg.prior_B_pos, a * cfg.prior_B_pos,
                              a * cfg.prior_B_dir, a * cfg.prior_B_dir};
        // Sigma^-1 = L^-T L^-1
        double Sinv[5][5];
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double s = 0.0;
                for (int m = (i > j ? i : j); m < 5; ++m) s += Li[pk(m, i)] * Li[pk(m, j)];
                Sinv[i][j] = s;
            }
        double logdet = 0.0, trBS = 0.0;
        for (int j = 0; j < 5; ++j) {
            logdet += 2.0 * log(L[pk(j, j)]);
            trBS += Bd[j] * Sinv[j][j];
        }
        const double pi = st.pi[rk];
        s_Fk[tid] = beta * q * log(pi) - 0.5 * beta * a * logdet - 0.5 * beta * trBS;
        if (dF != nullptr) {
            const double sc = dF[r];
            double* sk = s_st + tid * kStat;
            if (ystats) whitened_to_adjoint(Li, sk);
            const double invW = W > 0.0 ? 1.0 / W : 0.0;
            for (int c = 0; c < 5; ++c) g_delta[rk * 5 + c] = (float)(sc * sk[1 + c] * invW);
            for (int i = 0; i < 5; ++i)
                for (int j = 0; j <= i; ++j) {
                    double s = 0.0;   // (Sigma^-1 B L^-T)_{ij}
                    for (int c = 0; c <= j; ++c) s += Sinv[i][c] * Bd[c] * Li[pk(j, c)];
                    double gv = sk[6 + pk(i, j)] * invW + beta * s;
                    if (i == j) gv -= (sk[0] * invW + beta * a) / L[pk(i, i)];
                    g_L[rk * 15 + pk(i, j)] = (float)(sc * gv);
                }
            g_logit[rk] = (float)(sc * (sk[0] * invW - pi + beta * q * (1.0 - K * pi)));
        }
    }
    __syncthreads();
    if (tid == 0) {
        double F = W > 0.0 ? s_st[K * kStat + 1] / W : 0.0;
        for (int kk = 0; kk < K; ++kk) F += s_Fk[kk];
        if (F_out != nullptr) F_out[r] = F;
    }
}

// ---------------------------------------------------------------------------
// Initialisation (Sec. 4.3 "Initialization", App. B, App. C), one CTA per
// region.  The weighted picks are sums in sample order with explicit
// round-to-nearest FP64 operations (no contraction), so that the chosen
// samples are reproducible bit for bit: the CTA computes the weights of a
// chunk of samples in parallel and one thread adds them in order.
constexpr int kInitThreads = 128, kInitChunk = 8 * kInitThreads;

__device__ __forceinline__ double pick_weight(const float* __restrict__ pw, const float* __restrict__ px,
                                              const float* __restrict__ py, const float* __restrict__ pz,
                                              int64_t o, int64_t i, const int64_t* seeds, int n_seeds) {
    double c = (double)pw[o + i];
    c = c < 0.1 ? 0.1 : (c > 3.0 ? 3.0 : c);   // App. C: clamp to [W0, W1]
    if (n_seeds == 0) return c;
    double dmin = INFINITY;
    for (int s = 0; s < n_seeds; ++s) {
        const double dx = __dsub_rn((double)px[o + i], (double)px[o + seeds[s]]);
        const double dy = __dsub_rn((double)py[o + i], (double)py[o + seeds[s]]);
        const double dz = __dsub_rn((double)pz[o + i], (double)pz[o + seeds[s]]);
        const double dd = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        dmin = dd < dmin ? dd : dmin;
    }
    return __dmul_rn(c, dmin);
}

// the first i with u * sum(w) < w_0 + ... + w_i (the last positive weight if
// rounding leaves none), -1 if all weights vanish; every thread returns it
__device__ int64_t pick_index_cta(const float* __restrict__ pw, const float* __restrict__ px,
                                  const float* __restrict__ py, const float* __restrict__ pz, int64_t o,
                                  int64_t M, const int64_t* seeds, int n_seeds, double u, double* s_w,
                                  double* s_acc, int64_t* s_pick) {
    const int tid = threadIdx.x;
    // pass 1: the total, in sample order
    if (tid == 0) *s_acc = 0.0;
    for (int64_t c0 = 0; c0 < M; c0 += kInitChunk) {
        const int n = (int)min((int64_t)kInitChunk, M - c0);
        for (int q = tid; q < n; q += kInitThreads) s_w[q] = pick_weight(pw, px, py, pz, o, c0 + q, seeds, n_seeds);
        __syncthreads();
        if (tid == 0) {
            double a = *s_acc;
            for (int q = 0; q < n; ++q) a = __dadd_rn(a, s_w[q]);
            *s_acc = a;
        }
        __syncthreads();
    }
    const double tot = *s_acc;
    __syncthreads();
    if (!(tot > 0.0)) return -1;
    // pass 2: the first cumulative sum above u * total
    const double th = __dmul_rn(u, tot);
    if (tid == 0) {
        *s_acc = 0.0;
        s_pick[0] = -1;       // the answer
        s_pick[1] = -1;       // last index with a positive weight
    }
    __syncthreads();
    for (int64_t c0 = 0; c0 < M; c0 += kInitChunk) {
        const int n = (int)min((int64_t)kInitChunk, M - c0);
        for (int q = tid; q < n; q += kInitThreads) s_w[q] = pick_weight(pw, px, py, pz, o, c0 + q, seeds, n_seeds);
        __syncthreads();
        if (tid == 0) {
            double a = *s_acc;
            for (int q = 0; q < n; ++q) {
                a = __dadd_rn(a, s_w[q]);
                if (s_w[q] > 0.0) s_pick[1] = c0 + q;
                if (th < a) {
                    s_pick[0] = c0 + q;
                    break;
                }
            }
            *s_acc = a;
        }
        __syncthreads();
        if (s_pick[0] >= 0) break;                    // (uniform: read after the barrier)
    }
    const int64_t r = s_pick[0] >= 0 ? s_pick[0] : s_pick[1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kInitThreads) k_init_regions(sdmm_config cfg, BatchDesc d,
                                                               const double* __restrict__ extent,
                                                               const double* __restrict__ uniforms, sdmm_state st) {
    __shared__ double s_w[kInitChunk];
    __shared__ double s_acc;
    __shared__ int64_t s_pick[2];
    __shared__ int64_t seeds[SDMM_MAX_K / 8 > 0 ? SDMM_MAX_K / 8 : 1];
    const int64_t r = blockIdx.x;
    const int tid = threadIdx.x;
    const int K = cfg.K;
    const int n_pos = (K % 8 == 0) ? K / 8 : 1;
    const int n_dir = K / n_pos;
    const int64_t o = d.offsets[r], M = d.offsets[r + 1] - d.offsets[r];
    if (tid == 0) {
        st.n_seen[r] = 0;
        st.step_j[r] = 0;
        st.Wbar[r] = 0.0;
    }
    for (int e = tid; e < K * 16; e += kInitThreads) {
        const int k = e / 16, p = e % 16;
        if (p == 15) st.S0[r * K + k] = 0.0;
        else st.S2[(r * K + k) * 15 + p] = 0.0;
    }
    if (!(o >= 0 && M >= 0 && d.offsets[r + 1] <= d.N)) {
        if (tid == 0) st.status[r] = SDMM_REGION_BAD_OFFSETS;
        return;
    }
    if (M < cfg.min_samples || M <= 0) {
        if (tid == 0) st.status[r] = SDMM_REGION_SKIPPED;
        return;
    }
    const float* px = d.p[0];
    const float* py = d.p[1];
    const float* pz = d.p[2];
    const float* pw = d.p[6];
    for (int j = 0; j < n_pos; ++j) {
        const int64_t s = pick_index_cta(pw, px, py, pz, o, M, seeds, j, uniforms[r * n_pos + j], s_w, &s_acc, s_pick);
        if (tid == 0) seeds[j] = (s < 0) ? (j > 0 ? seeds[0] : 0) : s;
        __syncthreads();
    }
    const double rst = 2.0 * extent[r] / n_pos;            // App. B: r_st = 2 d / n_pos
    const double sx = rst / sqrt(kChi2_3_q90);
    const double sw = sqrt(kTwoPi / n_dir);                  // App. B: sigma^2 = 2 pi / n_dir
    for (int kk = tid; kk < K; kk += kInitThreads) {
        const int j = kk / n_dir, t = kk % n_dir;
        const int64_t rk = r * K + kk;
        double dv[3];
        if (n_dir == 8) {
            const double hh = 1.0 / sqrt(3.0);
            dv[0] = (t & 1) ? -hh : hh;
            dv[1] = (t & 2) ? -hh : hh;
            dv[2] = (t & 4) ? -hh : hh;
        } else {
            const double ga = 3.141592653589793238462643383279502884 * (3.0 - sqrt(5.0));
            const double z = 1.0 - (2.0 * t + 1.0) / n_dir;
            const double rad = sqrt(1.0 - z * z);
            dv[0] = rad * cos(ga * t);
            dv[1] = rad * sin(ga * t);
            dv[2] = z;
        }
        double mx[3] = {(double)px[o + seeds[j]], (double)py[o + seeds[j]], (double)pz[o + seeds[j]]};
        double L[15];
        for (int p = 0; p < 15; ++p) L[p] = 0.0;
        for (int c = 0; c < 3; ++c) L[pk(c, c)] = sx;
        for (int c = 3; c < 5; ++c) L[pk(c, c)] = sw;
        st.pi[rk] = 1.0 / K;
        for (int c = 0; c < 3; ++c) {
            st.mu_x[rk * 3 + c] = mx[c];
            st.mu_w[rk * 3 + c] = dv[c];
        }
        for (int p = 0; p < 15; ++p) st.L[rk * 15 + p] = L[p];
        write_records(1.0 / K, mx, dv, L, st.etab + rk * kE, st.qtab + rk * kQ, nullptr,
                      cfg.dir_coords == SDMM_DIR_EUCLIDEAN);
    }
    if (tid == 0) st.status[r] = SDMM_REGION_OK;
}

// ---------------------------------------------------------------------------
__global__ void k_prepare(int K, int64_t R, sdmm_state st, const double* __restrict__ logits,
                          const double* __restrict__ delta, int euclid) {
    const int64_t rk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rk >= R * K) return;
    if (logits != nullptr) {
        // pi = softmax(logits) over the region's K components
        const int64_t r0 = (rk / K) * K;
        double mx = -INFINITY;
        for (int kk = 0; kk < K; ++kk) mx = fmax(mx, logits[r0 + kk]);
        double s = 0.0;
        for (int kk = 0; kk < K; ++kk) s += exp(logits[r0 + kk] - mx);
        st.pi[rk] = exp(logits[rk] - mx) / s;
    }
    double mx[3], mw[3], L[15];
    for (int c = 0; c < 3; ++c) {
        mx[c] = st.mu_x[rk * 3 + c];
        mw[c] = st.mu_w[rk * 3 + c];
    }
    for (int p = 0; p < 15; ++p) L[p] = st.L[rk * 15 + p];
    write_records(st.pi[rk], mx, mw, L, st.etab + rk * kE, st.qtab + rk * kQ,
                  delta != nullptr ? delta + rk * 5 : nullptr, euclid != 0);
}

// ---------------------------------------------------------------------------
// Input validation: counts of samples whose direction is not unit length
// within tol, whose weight is negative or not finite, or whose position is
// not finite (three int64 counters, accumulated per CTA, then once per CTA).
__global__ void __launch_bounds__(256) k_validate(BatchDesc d, int64_t N, float tol,
                                                  unsigned long long* __restrict__ counts) {
    __shared__ unsigned int s_c[3];
    if (threadIdx.x < 3) s_c[threadIdx.x] = 0u;
    __syncthreads();
    unsigned int c[3] = {0u, 0u, 0u};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float ox = d.p[3][i], oy = d.p[4][i], oz = d.p[5][i], w = d.p[6][i];
        const float n2 = ox * ox + oy * oy + oz * oz;
        c[0] += !(fabsf(n2 - 1.f) <= 2.f * tol);                 // |w|^2 - 1 ~ 2 (|w| - 1)
        c[1] += !(w >= 0.f && isfinite(w));
        c[2] += !(isfinite(d.p[0][i]) && isfinite(d.p[1][i]) && isfinite(d.p[2][i]));
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        unsigned int v = c[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_c[q], v);
    }
    __syncthreads();
    if (threadIdx.x < 3 && s_c[threadIdx.x]) atomicAdd(counts + threadIdx.x, (unsigned long long)s_c[threadIdx.x]);
}

cudaError_t launch_validate(cudaStream_t s, const BatchDesc& d, int64_t N, float tol, unsigned long long* counts,
                            int grid) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || N == 0) return e;
    k_validate<<<grid, 256, 0, s>>>(d, N, tol, counts);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (declared in kernels.h)
template <int MODE>
static cudaError_t launch_acc_mode(int KP, dim3 grid, cudaStream_t s, WsHeader* ws,
                                   const int64_t* cb, const int32_t* cr, const float* etab, int K,
                                   int chunk, int density, float* partial, int ps, int write_ll,
                                   const float* chart2, int euclid) {
#define SDMM_ACC_CASE(P)                                                                       \
    case P:                                                                                    \
        k_accumulate<P, MODE><<<grid, kWarps * 32, 0, s>>>(ws, cb, cr, etab, K, chunk, density, \
                                                          partial, ps, write_ll, chart2, euclid); \
        break;
    switch (KP) {
        SDMM_ACC_CASE(1)
        SDMM_ACC_CASE(2)
        SDMM_ACC_CASE(4)
        SDMM_ACC_CASE(8)
        SDMM_ACC_CASE(16)
        SDMM_ACC_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef SDMM_ACC_CASE
    return cudaGetLastError();
}

cudaError_t launch_set_desc(cudaStream_t s, WsHeader* ws, const BatchDesc& d) {
    k_set_desc<<<1, 1, 0, s>>>(ws, d);
    return cudaGetLastError();
}

cudaError_t launch_build_chunks(cudaStream_t s, WsHeader* ws, int64_t* cb, int32_t* cr, int64_t* units,
                                int chunk, int min_samples, int64_t max_chunks) {
    k_build_chunks<<<1, 1024, 0, s>>>(ws, cb, cr, units, chunk, min_samples, max_chunks);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(cudaStream_t s, int mode, int KP, int grid, WsHeader* ws,
                              const int64_t* cb, const int32_t* cr, const float* etab, int K,
                              int chunk, int density, float* partial, int ps, int write_ll,
                              const float* chart2, int euclid, int chart_offsets) {
    if (mode == MODE_FIT && estep_fast_supported(KP)) {
        const bool solid = density == SDMM_DENSITY_SOLID_ANGLE;
        const int variant = euclid ? ESTEP_EUCLID
                            : solid ? (chart_offsets ? ESTEP_SOLID_OFFSETS : ESTEP_SOLID)
                                    : (chart_offsets ? ESTEP_OFFSETS : ESTEP_CHART);
        return launch_estep_fast(s, KP, grid, ws, cb, cr, etab, K, chunk, partial, ps, write_ll, variant);
    }
    if (mode == MODE_FIT)
        return launch_acc_mode<MODE_FIT>(KP, dim3(grid), s, ws, cb, cr, etab, K, chunk, density,
                                         partial, ps, write_ll, nullptr, euclid);
    if (mode == MODE_TWO && estep_fast_supported(KP))
        return launch_estep_fast(s, KP, grid, ws, cb, cr, etab, K, chunk, partial, ps, 0,
                                 density == SDMM_DENSITY_SOLID_ANGLE ? ESTEP_TWO_SOLID : ESTEP_TWO, chart2);
    if (mode == MODE_TWO)
        return launch_acc_mode<MODE_TWO>(KP, dim3(grid), s, ws, cb, cr, etab, K, chunk, density,
                                         partial, ps, 0, chart2, 0);
    return launch_acc_mode<MODE_GRAD>(KP, dim3(grid), s, ws, cb, cr, etab, K, chunk, density,
                                      partial, ps, write_ll, nullptr, euclid);
}

cudaError_t launch_new_charts(cudaStream_t s, int64_t R, WsHeader* ws, const int64_t* cb,
                              const float* partial, int ps, const sdmm_config& cfg,
                              const sdmm_state& st, float* chart2, int ystats) {
    k_new_charts<<<(unsigned)R, 128, 0, s>>>(ws, cb, partial, ps, cfg, st, chart2, ystats);
    return cudaGetLastError();
}

cudaError_t launch_reduce_mstep(cudaStream_t s, int64_t R, WsHeader* ws, const int64_t* cb,
                                const float* partial, int ps, const sdmm_config& cfg,
                                const sdmm_state& st, int iter, const float* xref,
                                const float* partial2, int ps2, int threads, int ystats) {
    // one CTA per region: thread k < K updates component k, all threads share
    // the reduction of the unit partials.  The caller picks the width: one
    // warp when the regions outnumber what 128-thread CTAs keep resident
    // (the per-component thread needs about 156 registers), four warps (a
    // faster reduction of many units) for a few large regions.
    const unsigned g1 = (unsigned)R;
    if (xref != nullptr)
        k_reduce_mstep<true, false, 1><<<g1, threads, 0, s>>>(ws, cb, partial, ps, cfg, st, iter, xref,
                                                              nullptr, 0, 0, R);
    else if (threads == 32 && cfg.K <= 16) {
        // two regions per warp (lanes 0-15 and 16-31)
        const unsigned g2 = (unsigned)((R + 1) / 2);
        if (partial2 != nullptr)
            k_reduce_mstep<false, true, 2><<<g2, 32, 0, s>>>(ws, cb, partial, ps, cfg, st, iter, xref,
                                                             partial2, ps2, ystats, R);
        else
            k_reduce_mstep<false, false, 2><<<g2, 32, 0, s>>>(ws, cb, partial, ps, cfg, st, iter, xref,
                                                              nullptr, 0, ystats, R);
    } else if (partial2 != nullptr)
        k_reduce_mstep<false, true, 1><<<g1, threads, 0, s>>>(ws, cb, partial, ps, cfg, st, iter, xref,
                                                              partial2, ps2, ystats, R);
    else
        k_reduce_mstep<false, false, 1><<<g1, threads, 0, s>>>(ws, cb, partial, ps, cfg, st, iter, xref,
                                                               nullptr, 0, ystats, R);
    return cudaGetLastError();
}

cudaError_t launch_reduce_objective(cudaStream_t s, int64_t R, const WsHeader* ws,
                                    const int64_t* cb, const float* partial, int ps,
                                    const sdmm_config& cfg, const sdmm_state& st, double* F,
                                    const double* dF, float* gd, float* gL, float* ga, int ystats) {
    k_reduce_objective<<<(unsigned)R, 128, 0, s>>>(ws, cb, partial, ps, cfg, st, F, dF, gd, gL, ga, ystats);
    return cudaGetLastError();
}

cudaError_t launch_init(cudaStream_t s, int64_t R, const sdmm_config& cfg, const BatchDesc& d,
                        const double* extent, const double* uniforms, const sdmm_state& st) {
    k_init_regions<<<(unsigned)R, kInitThreads, 0, s>>>(cfg, d, extent, uniforms, st);
    return cudaGetLastError();
}

cudaError_t launch_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st,
                           const double* logits, const double* delta, int euclid) {
    const int64_t n = R * K;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    k_prepare<<<blocks, 128, 0, s>>>(K, R, st, logits, delta, euclid);
    return cudaGetLastError();
}

}  // namespace sdmm
