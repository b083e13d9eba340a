// tc_fit.cu -- tensor-core (tcgen05) kernels.
//
//  k_tc_selftest   D = A B^T for one 128-row tile through the same shared-
//                  memory layouts, descriptors, MMA issue, commit and TMEM
//                  read-out helpers that the contraction-form E-step uses.
//  k_tc_prepare    per component: the coefficient rows of the contraction
//                  form, from the FP64 parameters.
//  k_tc_estep      contraction-form E-step + statistics (see below).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace sdmm {

constexpr uint64_t kTcWaitNs = 2000000000ull;   // 2 s bound on any MMA wait

// variant bits: 0 swap the K-major offsets; 1 A MN-major; 2 B MN-major;
// 3 swap the MN-major offsets (BF16 only for MN-major)
constexpr int kSelftestSmem = 200 * 1024;

__global__ void __launch_bounds__(128) k_tc_selftest(int kind, int N, int Kd, const float* __restrict__ A,
                                                     const float* __restrict__ B, float* __restrict__ D,
                                                     int variant, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int esize = kind == 0 ? 2 : 4;
    const int a_mn = (variant >> 1) & 1, b_mn = (variant >> 2) & 1;
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * Kd * esize;
    for (int e = tid; e < 128 * Kd; e += 128) {
        const int row = e / Kd, k = e % Kd;
        const uint32_t o = a_mn ? tc::mnmajor_offset(row, k, 128) : tc::kmajor_offset(row, k, Kd, esize);
        if (kind == 0) *reinterpret_cast<__nv_bfloat16*>(sA + o) = __float2bfloat16_rn(A[e]);
        else *reinterpret_cast<float*>(sA + o) = tc::to_tf32(A[e]);
    }
    for (int e = tid; e < N * Kd; e += 128) {
        const int row = e / Kd, k = e % Kd;
        const uint32_t o = b_mn ? tc::mnmajor_offset(row, k, N) : tc::kmajor_offset(row, k, Kd, esize);
        if (kind == 0) *reinterpret_cast<__nv_bfloat16*>(sB + o) = __float2bfloat16_rn(B[e]);
        else *reinterpret_cast<float*>(sB + o) = tc::to_tf32(B[e]);
    }
    tc::fence_smem_to_async();
    uint32_t ncols = 32;
    while (ncols < (uint32_t)N) ncols <<= 1;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t td = tmem_base;
    if (tid == 0) {
        const int kstep = kind == 0 ? 16 : 8;
        // K-major: (leading, stride) = (between K blocks, between 8-row blocks);
        // MN-major: (between K blocks, between MN blocks) -- both confirmed on GB300
        auto offs = [&](int mn_major, int rows, uint32_t* lbo, uint32_t* sbo, uint32_t* adv) {
            if (!mn_major) {
                const uint32_t a = 128, b = 8u * Kd * esize;
                *lbo = (variant & 1) ? b : a;
                *sbo = (variant & 1) ? a : b;
                *adv = 256;
            } else {
                const uint32_t a = 128, b = (uint32_t)(rows >> 3) * 128;
                *lbo = (variant & 8) ? a : b;     // MN-major: leading offset between K blocks
                *sbo = (variant & 8) ? b : a;     //           stride offset between MN blocks
                *adv = 2 * b;
            }
        };
        uint32_t al, as, aa, bl, bs, ba;
        offs(a_mn, 128, &al, &as, &aa);
        offs(b_mn, N, &bl, &bs, &ba);
        const uint32_t idesc = tc::instr_desc(kind == 0 ? 1 : 2, 128, N, a_mn, b_mn);
        for (int s = 0; s < Kd / kstep; ++s) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + s * aa, al, as);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + s * ba, bl, bs);
            if (kind == 0) tc::mma_f16(td, ad, bd, idesc, s > 0);
            else tc::mma_tf32(td, ad, bd, idesc, s > 0);
        }
        tc::mma_commit(&bar);
    }
    bool ok = tc::mbar_wait_bounded(&bar, 0, kTcWaitNs);
    if (!ok) ok = tc::mbar_wait_bounded(&bar, 0, kTcWaitNs);   // drain before freeing TMEM
    tc::fence_after_sync();
    if (ok) {
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tc::tmem_ld16(td + ((uint32_t)(warp * 32) << 16) + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(int64_t)tid * N + c + i] = v[i];
        }
    } else if (tid == 0) {
        *status = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(td, ncols);
}

cudaError_t launch_tc_selftest(cudaStream_t s, int kind, int N, int Kd, const float* A, const float* B,
                               float* D, int variant, int* status) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSelftestSmem);
    if (e != cudaSuccess) return e;
    k_tc_selftest<<<1, 128, kSelftestSmem, s>>>(kind, N, Kd, A, B, D, variant, status);
    return cudaGetLastError();
}

// ===========================================================================
// Contraction form of the E-step (derived from Sec. 3.1 Eq. log and the
// 5-D Gaussian of Eq. em-ss-computation).  With A_k = [t_k; b_k] (the first
// two rows of R_mu) the log map is nu = g A_k w, g = theta / sin theta, so
// for d = (x' - mu'_k, nu) and Q_k = Sigma_k^-1:
//   l_k = c5_k - d^T Q_k d / 2 = T0 + g T1 + g^2 T2,
//   T0 = c5 - (x'-mu')^T Qxx (x'-mu') / 2     (quadratic in x')
//   T1 = -(x'-mu')^T (Qxv A) w               (bilinear in x', w)
//   T2 = -w^T (A^T Qvv A) w / 2               (quadratic in w)
// and (u, v, c) = R_mu w.  All six are linear in the 28 shared features
// phi = [1, x', vech(x'x'), w, w (x) x', vech(ww)] (x' = x - xref, a
// per-region reference point), so one tile of 128 samples needs
//   GEMM 1:  Phi (128 x 32) . C_r^T (32 x 6K)   -> (u, v, c, T0, T1, T2)_k
// then, per sample (one thread per TMEM lane), theta = atan2(|(u,v)|, c),
// g, l_k, the log-sum-exp and w r_k, and for the statistics
//   GEMM 2:  [w r | w r g | w r g^2]^T (3K x 128) . Phi (128 x 32)
// accumulated in TMEM over the whole work unit; its rows are turned into
// s0, s1, s2 in FP64 by the M-step kernel (features_to_stats).
//
// Split products: an operand v is stored as hi = round(v) and lo =
// round(v - hi) in the MMA format (BF16 or TF32), and a.b ~ a_hi b_hi +
// a_hi b_lo + a_lo b_hi (three MMAs, FP32 accumulation).
constexpr int kTile = 128;
constexpr int kPhiPad = 32;     // features padded to the MMA K granularity

// coefficient rows of component rk: ctab[rk][6][32] (u, v, c, T0, T1, T2)
__global__ void k_tc_prepare(int K, int64_t R, sdmm_state st, float* __restrict__ ctab,
                             float* __restrict__ xref) {
    const int64_t rk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rk >= R * K) return;
    const int64_t r = rk / K;
    const int k = (int)(rk % K);
    // reference point: FP32 mean of the region's spatial means
    float xr[3];
    for (int c = 0; c < 3; ++c) {
        double m = 0.0;
        for (int j = 0; j < K; ++j) m += st.mu_x[(r * K + j) * 3 + c];
        xr[c] = (float)(m / K);
    }
    if (k == 0) {
        for (int c = 0; c < 3; ++c) xref[r * 4 + c] = xr[c];
        xref[r * 4 + 3] = 0.f;
    }
    double mp[3], muw[3], L[15], Li[15];
    for (int c = 0; c < 3; ++c) {
        mp[c] = st.mu_x[rk * 3 + c] - (double)xr[c];
        muw[c] = st.mu_w[rk * 3 + c];
    }
    for (int p = 0; p < 15; ++p) L[p] = st.L[rk * 15 + p];
    lower_inverse5_f64(L, Li);
    double Q[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double s = 0.0;
            for (int m = (i > j ? i : j); m < 5; ++m) s += Li[pk(m, i)] * Li[pk(m, j)];
            Q[i][j] = s;
        }
    double t[3], b[3];
    basis_f64(muw, t, b);
    const double A[2][3] = {{t[0], t[1], t[2]}, {b[0], b[1], b[2]}};
    double M[3][3], N[3][3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) M[a][c] = Q[a][3] * A[0][c] + Q[a][4] * A[1][c];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            double s = 0.0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) s += A[i][p] * Q[3 + i][3 + j] * A[j][q];
            N[p][q] = s;
        }
    const double pi = st.pi[rk];
    double c5 = (pi > 0.0 ? log(pi) : -INFINITY) - 2.5 * kLog2Pi;
    for (int j = 0; j < 5; ++j) c5 -= log(L[pk(j, j)]);
    double row[6][kPhiPad];
    for (int i = 0; i < 6; ++i)
        for (int f = 0; f < kPhiPad; ++f) row[i][f] = 0.0;
    for (int c = 0; c < 3; ++c) {
        row[0][10 + c] = t[c];
        row[1][10 + c] = b[c];
        row[2][10 + c] = muw[c];
    }
    // T0 = c5 - (x'-mu')^T Qxx (x'-mu') / 2
    double qmm = 0.0, Qm[3];
    for (int a = 0; a < 3; ++a) {
        Qm[a] = Q[a][0] * mp[0] + Q[a][1] * mp[1] + Q[a][2] * mp[2];
        qmm += mp[a] * Qm[a];
    }
    row[3][0] = c5 - 0.5 * qmm;
    for (int a = 0; a < 3; ++a) row[3][1 + a] = Qm[a];
    const int V[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int v = 0; v < 6; ++v) {
        const int a = V[v][0], c = V[v][1];
        row[3][4 + v] = (a == c ? -0.5 : -1.0) * Q[a][c];
        row[5][22 + v] = (a == c ? -0.5 : -1.0) * N[a][c];   // T2 = -w^T N w / 2
    }
    // T1 = -(x'-mu')^T M w: feature w_p x'_q (column 13 + 3p + q) has -M[q][p]
    for (int p = 0; p < 3; ++p) {
        row[4][10 + p] = mp[0] * M[0][p] + mp[1] * M[1][p] + mp[2] * M[2][p];
        for (int q = 0; q < 3; ++q) row[4][13 + 3 * p + q] = -M[q][p];
    }
    float* out = ctab + rk * 6 * kPhiPad;
    for (int i = 0; i < 6; ++i)
        for (int f = 0; f < kPhiPad; ++f) out[i * kPhiPad + f] = (float)row[i][f];
}

// ---- shared-memory plan of k_tc_estep (byte offsets, 1024-aligned base)
template <int K, int PREC>
struct TcPlan {
    static constexpr bool kTf32 = PREC != SDMM_PREC_TC_3XBF16;    // GEMM 1 in TF32
    static constexpr bool kSplit1 = PREC != SDMM_PREC_TC_TF32;     // GEMM 1 split (3 products)
    static constexpr int kE1 = kTf32 ? 4 : 2;                      // GEMM 1 element size
    static constexpr int kNQ = 6 * K;                              // GEMM 1 columns
    static constexpr int kPhi1 = kTile * kPhiPad * kE1;            // one GEMM 1 feature tile
    static constexpr int kPhiB = kTile * kPhiPad * 2;              // one BF16 feature tile
    static constexpr int kC1 = kNQ * kPhiPad * kE1;                // one coefficient tile
    static constexpr int kA2 = kTile * kTile * 2;                  // one statistics operand
    static constexpr int oPhi1h = 0;
    static constexpr int oPhi1l = oPhi1h + kPhi1;
    static constexpr int oPhiBh = oPhi1l + (kSplit1 ? kPhi1 : 0);
    static constexpr int oPhiBl = oPhiBh + (kTf32 ? kPhiB : 0);    // BF16 copy only for TF32 GEMM 1
    static constexpr int oC1h = oPhiBl + (kTf32 ? kPhiB : 0);
    static constexpr int oC1l = oC1h + kC1;
    static constexpr int oA2h = oC1l + (kSplit1 ? kC1 : 0);
    static constexpr int oA2l = oA2h + kA2;
    static constexpr int kBytes = oA2l + kA2;
    static constexpr uint32_t kCols = (kNQ + 32 <= 128) ? 128 : 256;   // TMEM: D1 then D2
    static constexpr uint32_t kD2 = kNQ;                                 // D2 column offset
};

template <int E>
__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
    if (E == 2) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
        if (lo) *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(v - __bfloat162float(h));
    } else {
        const float h = tc::to_tf32(v);
        *reinterpret_cast<float*>(hi + off) = h;
        if (lo) *reinterpret_cast<float*>(lo + off) = tc::to_tf32(v - h);
    }
}

// 8 consecutive BF16 values (hi and lo parts) as two 16-byte stores
__device__ __forceinline__ void store8_split_bf16(unsigned char* hi, unsigned char* lo, uint32_t off,
                                                  const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const float2 pf = __bfloat1622float2(p);
        const __nv_bfloat162 q = __floats2bfloat162_rn(v[2 * i] - pf.x, v[2 * i + 1] - pf.y);
        h[i] = *reinterpret_cast<const uint32_t*>(&p);
        l[i] = *reinterpret_cast<const uint32_t*>(&q);
    }
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int K, int PREC>
__global__ void __launch_bounds__(128, 1)
    k_tc_estep(WsHeader* __restrict__ ws, const int64_t* __restrict__ chunk_base,
               const int32_t* __restrict__ chunk_region, const float* __restrict__ ctab,
               const float* __restrict__ xref, int chunk, float* __restrict__ partial, int ps,
               int write_ll) {
    using P = TcPlan<K, PREC>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar1, bar2;
    __shared__ uint32_t tmem_base;
    __shared__ int s_c, s_abort;
    __shared__ float s_red[2][4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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

    unsigned char* sPhi1h = smem + P::oPhi1h;
    unsigned char* sPhi1l = P::kSplit1 ? smem + P::oPhi1l : nullptr;
    unsigned char* sPhiBh = P::kTf32 ? smem + P::oPhiBh : smem + P::oPhi1h;
    unsigned char* sPhiBl = P::kTf32 ? smem + P::oPhiBl : smem + P::oPhi1l;
    unsigned char* sC1h = smem + P::oC1h;
    unsigned char* sC1l = P::kSplit1 ? smem + P::oC1l : nullptr;
    unsigned char* sA2h = smem + P::oA2h;
    unsigned char* sA2l = smem + P::oA2l;

    // rows 3K..127 of the statistics operand stay zero
    for (int e = tid * 16; e < P::kA2; e += kTile * 16) {
        *reinterpret_cast<uint4*>(sA2h + e) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sA2l + e) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, P::kCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar1, 1);
        tc::mbar_init(&bar2, 1);
        tc::fence_mbar_init();
        s_abort = 0;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t td = tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

    // descriptors: GEMM 1 (K-major features x K-major coefficients)
    constexpr uint32_t g1_lbo = 128, g1_sbo = 8u * kPhiPad * P::kE1;
    constexpr int g1_k = P::kTf32 ? 8 : 16;
    constexpr int g1_steps = kPhiPad / g1_k;
    const uint32_t idesc1 = tc::instr_desc(P::kTf32 ? 2 : 1, kTile, P::kNQ);
    // GEMM 2 (MN-major statistics operand x MN-major BF16 features)
    constexpr uint32_t a2_lbo = (kTile / 8) * 128, a2_sbo = 128;
    constexpr uint32_t b2_lbo = (kPhiPad / 8) * 128, b2_sbo = 128;
    const uint32_t idesc2 = tc::instr_desc(1, kTile, kPhiPad, 1, 1);

    uint32_t ph1 = 0, ph2 = 0;
    bool g1_pending = false, g2_pending = false;
    bool aborted = false;
    int prev_r = -1;
    float xr0 = 0.f, xr1 = 0.f, xr2 = 0.f;

    // bounded wait for the next completion of `bar`; on success the group is
    // no longer pending, on timeout it stays pending (drained before exit)
    auto wait_or_abort = [&](uint64_t* bar, uint32_t& ph, bool& pending) -> bool {
        const bool ok = tc::mbar_wait_bounded(bar, ph, kTcWaitNs);
        if (ok) {
            ph ^= 1u;
            pending = false;
        } else if (tid == 0) {
            s_abort = 1;
            atomicExch(&ws->err, 1);
        }
        return ok;
    };

    for (;;) {
        if (tid == 0) s_c = atomicAdd(&ws->queue, 1);
        __syncthreads();
        const int c = s_c;
        if (c >= n_chunks || s_abort) break;
        const int r = chunk_region[c];
        if (r < 0 || r >= R) {
            __syncthreads();
            continue;
        }
        const int64_t start = off[r] + ((int64_t)c - chunk_base[r]) * chunk;
        const int64_t end = min(start + (int64_t)chunk, off[r + 1]);
        if (r != prev_r) {
            // coefficient tile of this region (no MMA reads it now: GEMM 1 of
            // the last tile has completed and GEMM 2 does not use it)
            prev_r = r;
            const float* cr = ctab + (int64_t)r * K * 6 * kPhiPad;
            for (int e = tid; e < P::kNQ * kPhiPad; e += kTile) {
                const int row = e / kPhiPad, f = e % kPhiPad;
                store_split<P::kE1>(sC1h, sC1l, tc::kmajor_offset(row, f, kPhiPad, P::kE1), __ldg(cr + e));
            }
            xr0 = __ldg(xref + r * 4 + 0);
            xr1 = __ldg(xref + r * 4 + 1);
            xr2 = __ldg(xref + r * 4 + 2);
        }
        float wsum = 0.f, wll = 0.f;
        bool first = true;
        for (int64_t g0 = start; g0 < end; g0 += kTile) {
            // statistics product of the previous tile must be done with Phi and A2
            if (g2_pending) {
                if (!wait_or_abort(&bar2, ph2, g2_pending)) aborted = true;
                tc::fence_after_sync();
            }
            if (__syncthreads_or(aborted)) { aborted = true; break; }
            // ---- features of sample g0 + tid (zero weight past the end)
            const int64_t i = g0 + tid;
            const bool valid = i < end;
            float x0 = 0.f, x1 = 0.f, x2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 1.f, wt = 0.f;
            if (valid) {
                x0 = __ldg(px + i) - xr0;
                x1 = __ldg(py + i) - xr1;
                x2 = __ldg(pz + i) - xr2;
                w0 = __ldg(ox + i);
                w1 = __ldg(oy + i);
                w2 = __ldg(oz + i);
                wt = __ldg(pw + i);
            }
            float phi[kPhiPad] = {1.f, x0, x1, x2, x0 * x0, x0 * x1, x0 * x2, x1 * x1, x1 * x2, x2 * x2,
                                  w0, w1, w2, w0 * x0, w0 * x1, w0 * x2, w1 * x0, w1 * x1, w1 * x2,
                                  w2 * x0, w2 * x1, w2 * x2, w0 * w0, w0 * w1, w0 * w2, w1 * w1, w1 * w2,
                                  w2 * w2, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int fb = 0; fb < kPhiPad; fb += 8) {
                store8_split_bf16(sPhiBh, sPhiBl, tc::kmajor_offset(tid, fb, kPhiPad, 2), phi + fb);
                if (P::kTf32) {
#pragma unroll
                    for (int f = fb; f < fb + 8; ++f)
                        store_split<4>(sPhi1h, sPhi1l, tc::kmajor_offset(tid, f, kPhiPad, 4), phi[f]);
                }
            }
            tc::fence_smem_to_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            // ---- GEMM 1
            if (tid == 0) {
                const uint32_t a_h = tc::smem_addr(sPhi1h), b_h = tc::smem_addr(sC1h);
                const uint32_t a_l = P::kSplit1 ? tc::smem_addr(sPhi1l) : 0u;
                const uint32_t b_l = P::kSplit1 ? tc::smem_addr(sC1l) : 0u;
                const int passes = P::kSplit1 ? 3 : 1;
                int n = 0;
                for (int pass = 0; pass < passes; ++pass) {
                    const uint32_t a = pass == 2 ? a_l : a_h;
                    const uint32_t b = pass == 1 ? b_l : b_h;
                    for (int s = 0; s < g1_steps; ++s, ++n) {
                        const uint64_t ad = tc::smem_desc(a + s * 256, g1_lbo, g1_sbo);
                        const uint64_t bd = tc::smem_desc(b + s * 256, g1_lbo, g1_sbo);
                        if (P::kTf32) tc::mma_tf32(td, ad, bd, idesc1, n > 0);
                        else tc::mma_f16(td, ad, bd, idesc1, n > 0);
                    }
                }
                tc::mma_commit(&bar1);
            }
            g1_pending = true;
            if (!wait_or_abort(&bar1, ph1, g1_pending)) aborted = true;
            tc::fence_after_sync();
            if (__syncthreads_or(aborted)) { aborted = true; break; }
            // ---- per-sample epilogue: theta, g, l_k, log-sum-exp, w r_k
            float lk[K], gk[K];
#pragma unroll
            for (int kb = 0; kb < K; kb += 8) {
                float v[48];
                tc::tmem_ld16(td + lane_base + 6 * kb, v);
                tc::tmem_ld16(td + lane_base + 6 * kb + 16, v + 16);
                tc::tmem_ld16(td + lane_base + 6 * kb + 32, v + 32);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float u = v[6 * j], vv = v[6 * j + 1], cz = v[6 * j + 2];
                    const float s2 = u * u + vv * vv;
                    const float rs = rsqrtf(s2);
                    const float th = atan2_pos(s2 * rs, cz);
                    const bool off_centre = s2 > 0.f;
                    const float g = off_centre ? th * rs : 1.f;
                    float l = v[6 * j + 3] + g * (v[6 * j + 4] + g * v[6 * j + 5]);
                    if (!off_centre && cz < 0.f) l = -INFINITY;
                    lk[kb + j] = l;
                    gk[kb + j] = g;
                }
            }
            float mx = lk[0];
#pragma unroll
            for (int k = 1; k < K; ++k) mx = fmaxf(mx, lk[k]);
            float se = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                lk[k] = (mx == -INFINITY) ? 0.f : __expf(lk[k] - mx);
                se += lk[k];
            }
            const float scale = se > 0.f ? wt / se : 0.f;
            const float li = se > 0.f ? mx + __logf(se) : -INFINITY;
            wsum += wt;
            wll += (wt > 0.f) ? wt * li : 0.f;
            if (loglik != nullptr && valid) loglik[i] = li;
            // statistics operand: rows k (w r), K + k (w r g), 2K + k (w r g^2)
#pragma unroll
            for (int kb = 0; kb < K; kb += 8) {
                float a8[8], b8[8], c8[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float wr = lk[kb + j] * scale;
                    a8[j] = wr;
                    b8[j] = wr * gk[kb + j];
                    c8[j] = b8[j] * gk[kb + j];
                }
                store8_split_bf16(sA2h, sA2l, tc::mnmajor_offset(kb, tid, kTile), a8);
                store8_split_bf16(sA2h, sA2l, tc::mnmajor_offset(K + kb, tid, kTile), b8);
                store8_split_bf16(sA2h, sA2l, tc::mnmajor_offset(2 * K + kb, tid, kTile), c8);
            }
            tc::fence_smem_to_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            // ---- GEMM 2 (accumulates over the work unit)
            if (tid == 0) {
                const uint32_t ah = tc::smem_addr(sA2h), al = tc::smem_addr(sA2l);
                const uint32_t bh = tc::smem_addr(sPhiBh), bl = tc::smem_addr(sPhiBl);
                int n = 0;
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t a = pass == 2 ? al : ah;
                    const uint32_t b = pass == 1 ? bl : bh;
                    for (int s = 0; s < kTile / 16; ++s, ++n) {
                        const uint64_t ad = tc::smem_desc(a + s * 2 * a2_lbo, a2_lbo, a2_sbo);
                        const uint64_t bd = tc::smem_desc(b + s * 2 * b2_lbo, b2_lbo, b2_sbo);
                        tc::mma_f16(td + P::kD2, ad, bd, idesc2, (n > 0 || !first) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&bar2);
            }
            g2_pending = true;
            first = false;
        }
        if (__syncthreads_or(aborted)) { aborted = true; break; }
        // ---- unit statistics: rows 0..3K-1 of D2, plus W and sum w l
        if (g2_pending) {
            if (!wait_or_abort(&bar2, ph2, g2_pending)) aborted = true;
            tc::fence_after_sync();
        }
        if (__syncthreads_or(aborted)) { aborted = true; break; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
            wll += __shfl_xor_sync(0xffffffffu, wll, o);
        }
        if (lane == 0) {
            s_red[0][warp] = wsum;
            s_red[1][warp] = wll;
        }
        if (warp * 32 < 3 * K) {
            float d[32];
            tc::tmem_ld16(td + lane_base + P::kD2, d);
            tc::tmem_ld16(td + lane_base + P::kD2 + 16, d + 16);
            if (tid < 3 * K) {
                float* out = partial + (int64_t)c * ps + tid * kFeat;
#pragma unroll
                for (int f = 0; f < kFeat; ++f) out[f] = d[f];
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            partial[(int64_t)c * ps + 3 * K * kFeat] = s_red[0][0] + s_red[0][1] + s_red[0][2] + s_red[0][3];
            partial[(int64_t)c * ps + 3 * K * kFeat + 1] = s_red[1][0] + s_red[1][1] + s_red[1][2] + s_red[1][3];
        }
    }
    // drain every product still in flight (after a timeout) before freeing TMEM
    if (g1_pending && !tc::mbar_wait_bounded(&bar1, ph1, kTcWaitNs) && tid == 0) atomicExch(&ws->err, 1);
    if (g2_pending && !tc::mbar_wait_bounded(&bar2, ph2, kTcWaitNs) && tid == 0) atomicExch(&ws->err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(td, P::kCols);
}

size_t tc_smem_bytes(int K, int prec) {
#define SDMM_TC_BYTES(KK, PP) \
    if (K == KK && prec == PP) return (size_t)TcPlan<KK, PP>::kBytes;
    SDMM_TC_BYTES(16, SDMM_PREC_TC_3XBF16) SDMM_TC_BYTES(16, SDMM_PREC_TC_TF32)
    SDMM_TC_BYTES(16, SDMM_PREC_TC_3XTF32) SDMM_TC_BYTES(32, SDMM_PREC_TC_3XBF16)
    SDMM_TC_BYTES(32, SDMM_PREC_TC_TF32) SDMM_TC_BYTES(32, SDMM_PREC_TC_3XTF32)
#undef SDMM_TC_BYTES
    return 0;
}

int tc_ctas_per_sm(int K, int prec) {
    const size_t b = tc_smem_bytes(K, prec) + 2048;            // + static shared memory
    const uint32_t cols = (6 * K + 32 <= 128) ? 128 : 256;
    int n = (int)((227u * 1024u) / b);
    n = n < (int)(512 / cols) ? n : (int)(512 / cols);
    return n < 1 ? 1 : n;
}

cudaError_t launch_tc_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st, float* ctab,
                              float* xref) {
    const int64_t n = R * K;
    k_tc_prepare<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(K, R, st, ctab, xref);
    return cudaGetLastError();
}

template <int K, int PREC>
static cudaError_t launch_tc_estep_t(cudaStream_t s, int grid, WsHeader* ws, const int64_t* cb,
                                     const int32_t* cr, const float* ctab, const float* xref, int chunk,
                                     float* partial, int ps, int write_ll) {
    const int bytes = TcPlan<K, PREC>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(k_tc_estep<K, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    k_tc_estep<K, PREC><<<grid, kTile, bytes, s>>>(ws, cb, cr, ctab, xref, chunk, partial, ps, write_ll);
    return cudaGetLastError();
}

cudaError_t launch_tc_estep(cudaStream_t s, int K, int prec, int grid, WsHeader* ws, const int64_t* cb,
                            const int32_t* cr, const float* ctab, const float* xref, int chunk,
                            float* partial, int ps, int write_ll) {
#define SDMM_TC_CASE(KK, PP)                                                                      \
    if (K == KK && prec == PP)                                                                    \
        return launch_tc_estep_t<KK, PP>(s, grid, ws, cb, cr, ctab, xref, chunk, partial, ps, write_ll);
    SDMM_TC_CASE(16, SDMM_PREC_TC_3XBF16) SDMM_TC_CASE(16, SDMM_PREC_TC_TF32)
    SDMM_TC_CASE(16, SDMM_PREC_TC_3XTF32) SDMM_TC_CASE(32, SDMM_PREC_TC_3XBF16)
    SDMM_TC_CASE(32, SDMM_PREC_TC_TF32) SDMM_TC_CASE(32, SDMM_PREC_TC_3XTF32)
#undef SDMM_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace sdmm
