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
// 3 swap the MN-major offsets (BF16 only for MN-major); 4 M = 64 (the read-out
// then shows where the 64 accumulator rows sit among the 128 TMEM lanes)
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
    const int M = (variant & 16) ? 64 : 128;
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * Kd * esize;
    for (int e = tid; e < M * Kd; e += 128) {
        const int row = e / Kd, k = e % Kd;
        const uint32_t o = a_mn ? tc::mnmajor_offset(row, k, M) : tc::kmajor_offset(row, k, Kd, esize);
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
        offs(a_mn, M, &al, &as, &aa);
        offs(b_mn, N, &bl, &bs, &ba);
        const uint32_t idesc = tc::instr_desc(kind == 0 ? 1 : 2, M, N, a_mn, b_mn);
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

// The bounded mbarrier wait of the E-step on a barrier that completes only if
// `arrive` is set: with nobody arriving the wait gives up after limit_ns and
// the kernel reports it (status 1) and returns normally.
__global__ void __launch_bounds__(128) k_wait_selftest(uint64_t limit_ns, int arrive, int* __restrict__ status,
                                                       unsigned long long* __restrict__ elapsed_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) tc::mbar_arrive(&bar);
    const uint64_t t0 = tc::global_ns();
    const bool ok = tc::mbar_wait_bounded(&bar, 0, limit_ns);
    const uint64_t dt = tc::global_ns() - t0;
    const int fail = __syncthreads_or(!ok);
    if (threadIdx.x == 0) {
        *status = fail ? 1 : 0;
        *elapsed_ns = (unsigned long long)dt;
    }
}

cudaError_t launch_wait_selftest(cudaStream_t s, uint64_t limit_ns, int arrive, int* status,
                                 unsigned long long* elapsed_ns) {
    k_wait_selftest<<<1, 128, 0, s>>>(limit_ns, arrive, status, elapsed_ns);
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
constexpr double kLog2E = 1.4426950408889634074;
constexpr float kLn2 = 0.693147180559945309f;

// coefficient rows of component rk: ctab[rk][6][32] (u, v, c, T0, T1, T2),
// the last three scaled by log2(e)
__global__ void k_tc_prepare(int K, int64_t R, sdmm_state st, float* __restrict__ ctab,
                             float* __restrict__ xref, int euclid) {
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
    if (euclid) {   // Euclidean ablation: unit rows, nu = A w - (mu_x, mu_y), g = 1
        t[0] = 1.0, t[1] = 0.0, t[2] = 0.0;
        b[0] = 0.0, b[1] = 1.0, b[2] = 0.0;
    } else {
        basis_f64(muw, t, b);
    }
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
    // a component of zero weight keeps a finite, negligible constant: an
    // infinite one would turn the split-product low part into NaN
    c5 = fmax(c5, -1e30);
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
    if (euclid) {
        // the offset o of nu = A w - o adds (x'-mu')^T Q_xn o - o^T Q_nn o / 2 to T0 and
        // w^T A^T Q_nn o to T1 (the kernel sums T0 + T1 + T2 with g = 1)
        const double o[2] = {muw[0], muw[1]};
        double wo[3], ono = 0.0;
        for (int a = 0; a < 3; ++a) wo[a] = Q[a][3] * o[0] + Q[a][4] * o[1];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) ono += o[i] * Q[3 + i][3 + j] * o[j];
        row[3][0] += -(mp[0] * wo[0] + mp[1] * wo[1] + mp[2] * wo[2]) - 0.5 * ono;
        for (int a = 0; a < 3; ++a) row[3][1 + a] += wo[a];
        for (int p = 0; p < 3; ++p)
            for (int i = 0; i < 2; ++i) row[4][10 + p] += A[i][p] * (Q[3 + i][3] * o[0] + Q[3 + i][4] * o[1]);
    }
    // T0, T1, T2 are stored times log2(e): the kernel's log-sum-exp runs in base 2
    for (int i = 3; i < 6; ++i)
        for (int f = 0; f < kPhiPad; ++f) row[i][f] *= kLog2E;
    float* out = ctab + rk * 6 * kPhiPad;
    for (int i = 0; i < 6; ++i)
        for (int f = 0; f < kPhiPad; ++f) out[i * kPhiPad + f] = (float)row[i][f];
}

// ---- k_tc_estep: a software-pipelined persistent kernel of 8 warps per CTA
// (two CTAs per SM where shared memory allows).  Warp w reads TMEM lane
// quadrant q = w % 4 (samples 32q..32q+31 of a tile) and owns component
// group h = w / 4 (K/2 components), so the two warps of a quadrant split the
// components of the same 32 samples.  Tiles of 128 samples flow through
//   phase A(t): load samples of tile t+2; features of tile t+1; issue GEMM
//               2(t-1); wait GEMM 1(t); l_k of tile t (own components) with
//               a local max and sum for the log-sum-exp
//   phase B(t): issue GEMM 1(t+1); merge the two groups' (max, sum); w r_k;
//               wait GEMM 2(t-1); statistics operand of tile t
// Warps meet only in pairs (the two warps of a quadrant, on a named
// barrier); operands reach the issuing lanes (warp 5: GEMM 1, warp 4: GEMM 2)
// through mbarrier arrivals of all eight warps, and products complete through
// tcgen05.commit mbarriers, so both products run while the CUDA cores work on
// the neighbouring tiles.  TMEM holds two GEMM 1 accumulators (tiles t, t+1)
// and the GEMM 2 accumulator of the current work unit; the BF16 features are
// triple-buffered (GEMM 2 of tile t-1 and GEMM 1 of tile t+1 read them while
// tile t+2's are written), the TF32 features double-buffered.  Every wait is
// bounded; a timeout sets the workspace error flag and a CTA-wide abort flag
// that ends every other wait, and the CTA drains and stops.
constexpr int kTcGroups = 2;                   // component groups per sample
constexpr int kTcWarps = 4 * kTcGroups;
constexpr int kTcThreads = kTcWarps * 32;
constexpr int kTcStatic = 4096;                // static shared memory of k_tc_estep (about 3 KB used)

template <int K, int PREC>
struct TcPlan {
    static constexpr bool kTf32 = PREC == SDMM_PREC_TC_TF32 || PREC == SDMM_PREC_TC_3XTF32;   // GEMM 1 in TF32
    static constexpr bool kSplit1 = PREC != SDMM_PREC_TC_TF32;      // GEMM 1 split (3 or 6 products)
    static constexpr bool kThree = PREC == SDMM_PREC_TC_6XBF16;     // BF16 in three pieces
    static constexpr int kE1 = kTf32 ? 4 : 2;                       // GEMM 1 element size
    static constexpr int kNQ = 6 * K;                               // GEMM 1 columns
    static constexpr int kKG = K / kTcGroups;                       // components per warp group
    static constexpr int kM2 = (3 * K <= 64) ? 64 : 128;            // GEMM 2 rows (3K used)
    static constexpr int kHalfB = kTile * kPhiPad * 2;              // BF16 feature tile (hi or lo)
    static constexpr int kHalfT = kTile * kPhiPad * 4;              // TF32 feature tile (hi or lo)
    static constexpr int kPhiB = (kThree ? 3 : 2) * kHalfB;         // hi + lo (+ third piece)
    static constexpr int kPhiT = kTf32 ? (kSplit1 ? 2 : 1) * kHalfT : 0;
    static constexpr int kHalfC = kNQ * kPhiPad * kE1;              // coefficient tile (hi or lo)
    static constexpr int kC1 = (kThree ? 3 : kSplit1 ? 2 : 1) * kHalfC;
    static constexpr int kHalfA = kM2 * kTile * 2;                  // statistics operand (hi or lo)
    static constexpr int kA2 = 2 * kHalfA;
    static constexpr int kStage = 7 * kTile * 4;                    // one tile's samples (7 streams)
    static constexpr int kRest = 2 * kPhiT + kC1 + kA2 + 3 * kStage;
    // BF16 feature buffers: three when that leaves room for two CTAs per SM
    // (or for one), else two (the late store waits for GEMM 2(t-1))
    static constexpr bool fits2(int b) { return (b + kTcStatic + 1024) * 2 <= 228 * 1024; }
    static constexpr int kNB = fits2(3 * kPhiB + kRest) ? 3
                               : fits2(2 * kPhiB + kRest) ? 2
                               : 3 * kPhiB + kRest + kTcStatic <= 227 * 1024 ? 3 : 2;
    static constexpr bool kEarlyB = !kTf32 && kNB == 3;             // BF16 features stored before GEMM 1(t) ends
    static constexpr int oPhiB = 0;
    static constexpr int oPhiT = kNB * kPhiB;
    static constexpr int oC1 = oPhiT + 2 * kPhiT;
    static constexpr int oA2 = oC1 + kC1;
    static constexpr int oStage = oA2 + kA2;
    static constexpr int kBytes = oStage + 3 * kStage;
    static constexpr uint32_t kD2 = 2 * kNQ;                        // D1[0], D1[1], then D2
    static constexpr uint32_t kCols = kD2 + 32 <= 256 ? 256 : 512;
    static constexpr int kCtas = fits2(kBytes) && kCols * 2 <= 512 ? 2 : 1;
    static_assert(kBytes + kTcStatic <= 227 * 1024, "shared memory plan too large");
    static_assert(kTf32 || kEarlyB || kThree, "two-buffer BF16 plans are planned for the 6xBF16 form only");
    static_assert(kD2 + 32 <= 512, "TMEM plan too large");
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

// hi and lo BF16 parts of n = 4 or 8 consecutive values (one 8- or 16-byte store
// each), through 32-bit shared-window addresses
template <int N>
__device__ __forceinline__ void sts_split_bf16(uint32_t hi, uint32_t lo, const float* v) {
    uint32_t h[N / 2], l[N / 2];
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const float2 pf = __bfloat1622float2(p);
        const __nv_bfloat162 q = __floats2bfloat162_rn(v[2 * i] - pf.x, v[2 * i + 1] - pf.y);
        h[i] = *reinterpret_cast<const uint32_t*>(&p);
        l[i] = *reinterpret_cast<const uint32_t*>(&q);
    }
    if (N == 8) {
        tc::sts128(hi, h[0], h[1], h[2], h[3]);
        tc::sts128(lo, l[0], l[1], l[2], l[3]);
    } else {
        tc::sts64(hi, h[0], h[1]);
        tc::sts64(lo, l[0], l[1]);
    }
}
// three BF16 pieces of 8 consecutive values: p0 = bf16(v), p1 = bf16(v - p0),
// p2 = bf16(v - p0 - p1), so that v = p0 + p1 + p2 to about 2^-24 relative
__device__ __forceinline__ void sts_split3_bf16(uint32_t a0, uint32_t a1, uint32_t a2, const float* v) {
    uint32_t p0[4], p1[4], p2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const float2 hf = __bfloat1622float2(h);
        const float r0 = v[2 * i] - hf.x, r1 = v[2 * i + 1] - hf.y;
        const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
        const float2 mf = __bfloat1622float2(m);
        const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
        p0[i] = *reinterpret_cast<const uint32_t*>(&h);
        p1[i] = *reinterpret_cast<const uint32_t*>(&m);
        p2[i] = *reinterpret_cast<const uint32_t*>(&l);
    }
    tc::sts128(a0, p0[0], p0[1], p0[2], p0[3]);
    tc::sts128(a1, p1[0], p1[1], p1[2], p1[3]);
    tc::sts128(a2, p2[0], p2[1], p2[2], p2[3]);
}
// hi (and, if LO, lo) TF32 parts of 4 consecutive values (16-byte stores)
template <bool LO>
__device__ __forceinline__ void sts_split_tf32(uint32_t hi, uint32_t lo, const float* v) {
    float h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = tc::to_tf32(v[i]);
        l[i] = tc::to_tf32(v[i] - h[i]);
    }
    tc::sts128(hi, __float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
    if (LO) tc::sts128(lo, __float_as_uint(l[0]), __float_as_uint(l[1]), __float_as_uint(l[2]), __float_as_uint(l[3]));
}


// A tile of up to 128 consecutive samples of one work unit.
struct TcTile {
    int64_t g0;         // first sample
    int c, r;           // unit, region (r < 0: no valid sample)
    int n;              // valid samples in the tile (0..128)
    bool first, live;   // first tile of its unit; tile exists
};

template <int K, int PREC, bool EU>
__global__ void __launch_bounds__(kTcThreads, TcPlan<K, PREC>::kCtas)
    k_tc_estep(WsHeader* __restrict__ ws, const int32_t* __restrict__ chunk_region,
               const int64_t* __restrict__ units, const float* __restrict__ ctab,
               const float* __restrict__ xref, float* __restrict__ partial, int ps, int write_ll,
               int solid) {
    using P = TcPlan<K, PREC>;
    constexpr int KG = P::kKG;
    constexpr int RPQ = P::kM2 / 4;                // GEMM 2 rows per TMEM lane quadrant
    extern __shared__ __align__(1024) unsigned char smem[];
    // bar1 / bar2: GEMM 1 / GEMM 2 completed; rdy1 / rdy2: their operands are
    // in shared memory (one arrival per warp)
    __shared__ __align__(8) uint64_t bar1, bar2, rdy1, rdy2;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float2 s_ml[kTcGroups][kTile];      // per group, per sample: (m, sum 2^(l_k log2 e - m))
    __shared__ float s_xr[3][4][4];                // per staging slot and quadrant: region reference point
    __shared__ const float* s_stream[7];           // the batch's sample streams (fixed for the launch)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, grp = warp >> 2;
    const int smp = quad * 32 + lane;              // sample (TMEM lane) of this thread

    unsigned char* const sC1h = smem + P::oC1;
    unsigned char* const sC1l = P::kSplit1 ? smem + P::oC1 + P::kHalfC : nullptr;
    unsigned char* const sA2h = smem + P::oA2;
    unsigned char* const sA2l = smem + P::oA2 + P::kHalfA;
    auto phiB = [&](int b) { return smem + P::oPhiB + b * P::kPhiB; };
    auto phiT = [&](int b) { return smem + P::oPhiT + b * P::kPhiT; };

    // rows 3K..M2-1 of the statistics operand only reach accumulator rows
    // that are never read; they are cleared once all the same
    for (int e = tid * 16; e < P::kA2; e += kTcThreads * 16)
        *reinterpret_cast<uint4*>(sA2h + e) = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, P::kCols);
        tc::tmem_relinquish();
    }
    if (tid < 7) s_stream[tid] = ws->desc.p[tid];
    if (tid == 0) {
        tc::mbar_init(&bar1, 1);
        tc::mbar_init(&bar2, 1);
        tc::mbar_init(&rdy1, kTcWarps);
        tc::mbar_init(&rdy2, kTcWarps);
        tc::fence_mbar_init();
        s_abort = 0;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t td = tmem_base;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;

    // ---- work units of this CTA: a static round robin over the CTAs, walked
    // in the same order by every warp; the next unit's range is loaded one
    // unit ahead
    const int64_t n_chunks = ws->n_chunks;
    const int64_t R = ws->desc.R;
    int64_t uc = blockIdx.x;
    const int64_t u_end = n_chunks;
    int pr = -1;
    int64_t ps0 = 0, pe = 0, uend = 0;   // next unit's start / end; end of the unit being walked
    auto fetch = [&]() {
        if (uc < u_end) {
            pr = __ldg(chunk_region + uc);
            ps0 = __ldg(units + 2 * uc);
            pe = __ldg(units + 2 * uc + 1);
        }
    };
    auto enter = [&](TcTile& tl) {
        tl.live = uc < u_end;
        if (!tl.live) return;
        tl.c = (int)uc;
        tl.r = (pr >= 0 && pr < R) ? pr : -1;
        tl.g0 = ps0;
        uend = tl.r >= 0 ? pe : ps0;
        tl.n = (int)min((int64_t)kTile, uend - ps0);
        tl.first = true;
        uc += gridDim.x;
        fetch();
    };
    // only the walker furthest ahead calls this; the others copy its tiles
    auto advance = [&](TcTile& tl) {
        if (!tl.live) return;
        if (tl.g0 + kTile < uend) {
            tl.g0 += kTile;
            tl.n = (int)min((int64_t)kTile, uend - tl.g0);
            tl.first = false;
        } else {
            enter(tl);
        }
    };
    fetch();

    // ---- bounded waits; a timeout anywhere stops every wait of the CTA
    bool aborted = false;
    auto wait_bar = [&](uint64_t* b, uint32_t parity) -> bool {
        if (tc::mbar_try_wait(b, parity)) return true;
        const uint64_t t0 = tc::global_ns();
        while (true) {
            if (tc::mbar_try_wait_hint(b, parity, 100000u)) return true;   // suspends, no spinning
            if (*reinterpret_cast<volatile int*>(&s_abort)) return false;
            if (tc::global_ns() - t0 > kTcWaitNs) {
                *reinterpret_cast<volatile int*>(&s_abort) = 1;
                atomicExch(&ws->err, 1);
                return false;
            }
        }
    };
    uint32_t ph1 = 0, ph2 = 0, pr1 = 0, pr2 = 0;
    bool g1_pending = false, g2_pending = false;
    auto wait_mma = [&](uint64_t* b, uint32_t& ph, bool& pending) {
        if (!pending) return;
        if (wait_bar(b, ph)) {
            ph ^= 1u;
            pending = false;
        } else {
            aborted = true;
        }
        tc::fence_after_sync();
    };
    // this warp's shared-memory writes and TMEM reads are complete: one arrival on b
    auto signal = [&](uint64_t* b) {
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(b);
    };
    // barrier of the two warps of a quadrant (they share their 32 samples);
    // it also makes the abort decision common to both
    auto sync_pair = [&]() {
        tc::fence_before_sync();
        const bool p = aborted || *reinterpret_cast<volatile int*>(&s_abort);
        switch (quad) {                          // barrier ids 1..4, one per quadrant
            case 0: aborted = tc::bar_red_or<1, 64>(p); break;
            case 1: aborted = tc::bar_red_or<2, 64>(p); break;
            case 2: aborted = tc::bar_red_or<3, 64>(p); break;
            default: aborted = tc::bar_red_or<4, 64>(p); break;
        }
        tc::fence_after_sync();
    };

    // ---- MMA issue: one lane of warp 5 (GEMM 1) and of warp 4 (GEMM 2),
    // once every warp has signalled the operands
    constexpr uint32_t g1_sbo = 8u * kPhiPad * P::kE1;
    constexpr int g1_k = P::kTf32 ? 8 : 16;
    constexpr uint32_t a2_lbo = (P::kM2 / 8) * 128, b2_lbo = (kPhiPad / 8) * 128;
    // GEMM 1: K-major features x K-major coefficients (M = 128, N = 6K) into D1[t & 1]
    auto issue_g1 = [&](int t) {
        const bool ok = wait_bar(&rdy1, pr1);
        pr1 ^= 1u;
        tc::fence_after_sync();
        if (ok && lane == 0) {
            const uint64_t a0 = P::kTf32 ? tc::smem_desc(tc::smem_addr(phiT(t & 1)), 128, g1_sbo)
                                         : tc::smem_desc(tc::smem_addr(phiB(t % P::kNB)), 128, g1_sbo);
            constexpr uint32_t a_piece = P::kTf32 ? P::kHalfT : P::kHalfB;
            const uint32_t d = td + (uint32_t)(t & 1) * P::kNQ;
            const uint32_t idesc1 = tc::instr_desc(P::kTf32 ? 2 : 1, kTile, P::kNQ);
            const uint64_t b0 = tc::smem_desc(tc::smem_addr(sC1h), 128, g1_sbo);
            // products of pieces (i of the features, j of the coefficients):
            // split forms keep (0,0) (0,1) (1,0); three pieces also (0,2) (1,1) (2,0)
            constexpr int np = P::kThree ? 6 : P::kSplit1 ? 3 : 1;
            constexpr int pi_[6] = {0, 0, 1, 0, 1, 2}, pj_[6] = {0, 1, 0, 2, 1, 0};
            int n = 0;
#pragma unroll
            for (int pass = 0; pass < np; ++pass) {
                const uint64_t a = tc::desc_add(a0, pi_[pass] * a_piece);
                const uint64_t b = tc::desc_add(b0, pj_[pass] * P::kHalfC);
#pragma unroll
                for (int s = 0; s < kPhiPad / g1_k; ++s, ++n) {
                    if (P::kTf32) tc::mma_tf32(d, tc::desc_add(a, s * 256), tc::desc_add(b, s * 256), idesc1, n > 0);
                    else tc::mma_f16(d, tc::desc_add(a, s * 256), tc::desc_add(b, s * 256), idesc1, n > 0);
                }
            }
            tc::mma_commit(&bar1);
        }
        __syncwarp();
        if (!ok) aborted = true;
    };
    // GEMM 2: MN-major statistics operand (M = M2) x MN-major BF16 features
    // (N = 32), accumulated over the work unit
    auto issue_g2 = [&](int t, bool restart) {
        const bool ok = wait_bar(&rdy2, pr2);
        pr2 ^= 1u;
        tc::fence_after_sync();
        if (ok && lane == 0) {
            const uint64_t bh = tc::smem_desc(tc::smem_addr(phiB(t % P::kNB)), b2_lbo, 128);
            const uint64_t bl = tc::desc_add(bh, P::kHalfB);
            const uint32_t idesc2 = tc::instr_desc(1, P::kM2, kPhiPad, 1, 1);
            const uint64_t dA2h = tc::smem_desc(tc::smem_addr(sA2h), a2_lbo, 128);
            const uint64_t dA2l = tc::desc_add(dA2h, P::kHalfA);
            int n = 0;
#pragma unroll
            for (int pass = 0; pass < 3; ++pass) {
                const uint64_t a = pass == 2 ? dA2l : dA2h;
                const uint64_t b = pass == 1 ? bl : bh;
#pragma unroll
                for (int s = 0; s < kTile / 16; ++s, ++n)
                    tc::mma_f16(td + P::kD2, tc::desc_add(a, s * 2 * a2_lbo), tc::desc_add(b, s * 2 * b2_lbo),
                                idesc2, (n > 0 || !restart) ? 1u : 0u);
            }
            tc::mma_commit(&bar2);
        }
        __syncwarp();
        if (!ok) aborted = true;
    };

    float* __restrict__ loglik = write_ll ? ws->desc.loglik : nullptr;
    // Per-thread shared-window addresses of the hot loop (32-bit, fixed for
    // the whole kernel; buffers and slots are added as byte offsets)
    const uint32_t sbase = tc::smem_addr(smem);
    const uint32_t aPhiB = sbase + P::oPhiB + tc::kmajor_offset(smp, 16 * grp, kPhiPad, 2);   // +128: features 8..15
    const uint32_t aPhiT = sbase + P::oPhiT + tc::kmajor_offset(smp, 16 * grp, kPhiPad, 4);   // +128 per 4 features
    const uint32_t aA2 = sbase + P::oA2 + tc::mnmajor_offset(3 * KG * grp, smp, P::kM2);     // +128 per 8 rows
    const uint32_t aStage = sbase + P::oStage + smp * 4;   // + slot 7*128*4 + stream 128*4
    const uint32_t aML = tc::smem_addr(&s_ml[0][smp]);     // + group 128*8
    const uint32_t aXr = tc::smem_addr(&s_xr[0][quad][0]); // + slot 64
    constexpr uint32_t kSlot = 7 * kTile * 4, kStream = kTile * 4;
    // sample staging ring: slot s holds a tile's 7 streams [7][128] and its
    // region's reference point.  The two warps of a quadrant copy streams 0-3
    // (group 0, plus the reference point) and 4-6 (group 1) of their 32
    // samples; every thread waits for its own copies before the pair barrier
    // that ends phase B, after which the slot is read (one phase later).
    auto load = [&](const TcTile& tl, int slot) {
        const bool valid = tl.live && smp < tl.n;
        const int64_t i = valid ? tl.g0 + smp : 0;
        const uint32_t dst = aStage + slot * kSlot;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * grp + j;
            if (q < 7) tc::cp_async4s(dst + q * kStream, s_stream[q] + i, valid);
        }
        if (grp == 0 && lane < 3) {
            const bool rv = tl.live && tl.r >= 0;
            tc::cp_async4s(aXr + slot * 64 + lane * 4, xref + (rv ? tl.r * 4 + lane : 0), rv);
        }
        tc::cp_async_commit();
    };
    auto sample = [&](int slot, int q) { return tc::lds32(aStage + slot * kSlot + q * kStream); };
    // this group's 16 of the 32 features phi = [1, x', vech(x'x'), w, w (x) x', vech(ww)]
    auto features = [&](int slot, float* f) {
        const uint32_t xr = aXr + slot * 64;
        const float x0 = sample(slot, 0) - tc::lds32(xr), x1 = sample(slot, 1) - tc::lds32(xr + 4),
                    x2 = sample(slot, 2) - tc::lds32(xr + 8);
        const float w0 = sample(slot, 3), w1 = sample(slot, 4), w2 = sample(slot, 5);
        if (grp == 0) {
            f[0] = 1.f; f[1] = x0; f[2] = x1; f[3] = x2;
            f[4] = x0 * x0; f[5] = x0 * x1; f[6] = x0 * x2; f[7] = x1 * x1;
            f[8] = x1 * x2; f[9] = x2 * x2; f[10] = w0; f[11] = w1;
            f[12] = w2; f[13] = w0 * x0; f[14] = w0 * x1; f[15] = w0 * x2;
        } else {
            f[0] = w1 * x0; f[1] = w1 * x1; f[2] = w1 * x2; f[3] = w2 * x0;
            f[4] = w2 * x1; f[5] = w2 * x2; f[6] = w0 * w0; f[7] = w0 * w1;
            f[8] = w0 * w2; f[9] = w1 * w1; f[10] = w1 * w2; f[11] = w2 * w2;
            f[12] = 0.f; f[13] = 0.f; f[14] = 0.f; f[15] = 0.f;
        }
    };
    auto store_b = [&](int b, const float* f) {
        const uint32_t a = aPhiB + b * P::kPhiB;
        if constexpr (P::kThree) {
            sts_split3_bf16(a, a + P::kHalfB, a + 2 * P::kHalfB, f);
            sts_split3_bf16(a + 128, a + 128 + P::kHalfB, a + 128 + 2 * P::kHalfB, f + 8);
        } else {
            sts_split_bf16<8>(a, a + P::kHalfB, f);
            sts_split_bf16<8>(a + 128, a + 128 + P::kHalfB, f + 8);
        }
    };
    auto store_t = [&](int b, const float* f) {
        const uint32_t a = aPhiT + b * P::kPhiT;
#pragma unroll
        for (int h = 0; h < 4; ++h) sts_split_tf32<P::kSplit1>(a + 128 * h, a + 128 * h + P::kHalfT, f + 4 * h);
    };
    auto load_c1 = [&](int r) {
        const float* cr = ctab + (int64_t)r * K * 6 * kPhiPad;
        for (int e = tid; e < P::kNQ * kPhiPad; e += kTcThreads) {
            const int row = e / kPhiPad, f = e % kPhiPad;
            const uint32_t o = tc::kmajor_offset(row, f, kPhiPad, P::kE1);
            const float v = __ldg(cr + e);
            if constexpr (P::kThree) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                const float r0 = v - __bfloat162float(h);
                const __nv_bfloat16 m = __float2bfloat16_rn(r0);
                *reinterpret_cast<__nv_bfloat16*>(sC1h + o) = h;
                *reinterpret_cast<__nv_bfloat16*>(sC1h + P::kHalfC + o) = m;
                *reinterpret_cast<__nv_bfloat16*>(sC1h + 2 * P::kHalfC + o) =
                    __float2bfloat16_rn(r0 - __bfloat162float(m));
            } else {
                store_split<P::kE1>(sC1h, sC1l, o, v);
            }
        }
    };
    // unit statistics out of D2 (rows (h, j, kk) -> partial row j K + h KG + kk)
    // and, per quadrant, the unit's W and sum w l (summed by the M-step)
    float accW = 0.f, accL = 0.f;
    auto flush = [&](int c) {
        if (grp == 1 && quad * RPQ < 3 * K) {
            float d[32];
            tc::tmem_ld16(td + lane_base + P::kD2, d);
            tc::tmem_ld16(td + lane_base + P::kD2 + 16, d + 16);
            const int m = quad * RPQ + lane;
            if (lane < RPQ && m < 3 * K) {
                const int h = m / (3 * KG), j = (m % (3 * KG)) / KG, kk = m % KG;
                float* out = partial + (int64_t)c * ps + (j * K + h * KG + kk) * kFeat;
#pragma unroll
                for (int f = 0; f < kFeat; ++f) out[f] = d[f];
            }
        }
        if (grp == 0) {
            float a = accW, b = accL;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
            }
            if (lane == 0) {
                partial[(int64_t)c * ps + 3 * K * kFeat + quad] = a;
                partial[(int64_t)c * ps + 3 * K * kFeat + 4 + quad] = b;
            }
            accW = accL = 0.f;
        }
    };

    // ---- prologue: tile 0 through its GEMM 1
    TcTile cur, nxt, nn;
    enter(cur);
    if (cur.live) {
        load(cur, 0);
        nxt = cur;
        advance(nxt);
        load(nxt, 1);
        if (cur.r >= 0) load_c1(cur.r);
        float f[16];
        tc::cp_async_wait<0>();                  // tiles 0 and 1
        sync_pair();
        features(0, f);
        store_b(0, f);
        if (P::kTf32) store_t(0, f);
        signal(&rdy1);
        if (warp == 5) issue_g1(0);
        g1_pending = true;
    }
    int t = 0, prev_c = -1;
    int s0 = 0, s1 = 1, s2 = 2;                   // staging slots of tiles t, t+1, t+2
    int b1 = 1 % P::kNB;                          // BF16 feature buffer of tile t+1
    bool a2_ready = false, a2_restart = false;
    while (cur.live && !aborted) {
        // ---- phase A
        nn = nxt;
        advance(nn);
        load(nn, s2);                             // waited for at the end of phase B
        float f[16];
        if (nxt.live) {
            features(s1, f);
            if (P::kEarlyB) store_b(b1, f);
            else if (P::kTf32) store_t((t + 1) & 1, f);
        }
        if (a2_ready) {                           // GEMM 2 of the previous tile
            if (warp == 4) issue_g2(t - 1, a2_restart);
            g2_pending = true;
            a2_ready = false;
        }
        wait_mma(&bar1, ph1, g1_pending);         // GEMM 1(t)
        if (nxt.live && nxt.r >= 0 && nxt.r != cur.r) load_c1(nxt.r);
        // l_k log2(e) of this group's components: TMEM columns 6 (h KG + j) + (u, v, c, T0, T1, T2)
        float lk[KG], gk[KG];
        {
            auto eval1 = [&](const float* q, int j) {
                if constexpr (EU) {             // ablation: no change of variables, g = 1
                    lk[j] = q[3] + q[4] + q[5];
                    gk[j] = 1.f;
                    return;
                }
                const float u = q[0], vv = q[1], cz = q[2];
                const float s2 = u * u + vv * vv;
                const bool cut = s2 == 0.f && cz < 0.f;    // cut locus: undefined chart
                const float g = cut ? 1.f : g_of_cos(cz, tc::rsqrt_approx(s2));
                float l = q[3] + g * (q[4] + g * q[5]);
                // solid-angle density p^t / sinc |nu| (Sec. 3.1 Eq. solidangle-pdf):
                // + log2(theta / sin theta); the per-sample maximum below is exact
                if (solid) l += tc::lg2_approx(g);
                if (cut) l = -INFINITY;
                lk[j] = l;
                gk[j] = g;
            };
            // chunks of 8 components = 48 columns, starting on a multiple of 16
#pragma unroll
            for (int cb = 0; cb < KG; cb += 8) {
                const uint32_t col = (uint32_t)(t & 1) * P::kNQ + 6u * (KG * grp + cb);
                float v[48];
                tc::tmem_ld16(td + lane_base + col, v);
                tc::tmem_ld16(td + lane_base + col + 16, v + 16);
                tc::tmem_ld16(td + lane_base + col + 32, v + 32);
#pragma unroll
                for (int j = 0; j < 8; ++j) eval1(v + 6 * j, cb + j);
            }
        }
        float mg = lk[0];
#pragma unroll
        for (int j = 1; j < KG; ++j) mg = fmaxf(mg, lk[j]);
        float sg = 0.f;
#pragma unroll
        for (int j = 0; j < KG; ++j) {
            lk[j] = mg > -INFINITY ? tc::ex2_approx(lk[j] - mg) : 0.f;   // lk now holds 2^(l_k - m_h)
            sg += lk[j];
        }
        tc::sts64(aML + grp * kTile * 8, __float_as_uint(mg), __float_as_uint(sg));
        if (!P::kEarlyB && nxt.live) {
            if (P::kNB == 2) wait_mma(&bar2, ph2, g2_pending);   // GEMM 2(t-1) reads this buffer
            features(s1, f);
            store_b(b1, f);
        }
        if (nxt.live) signal(&rdy1);
        sync_pair();
        if (aborted) break;
        // ---- phase B
        if (nxt.live) {
            if (warp == 5) issue_g1(t + 1);
            g1_pending = true;
        }
        const float2 m0 = tc::lds64(aML), m1 = tc::lds64(aML + kTile * 8);
        const float M = fmaxf(m0.x, m1.x);
        const float e0 = m0.x > -INFINITY ? tc::ex2_approx(m0.x - M) : 0.f;
        const float e1 = m1.x > -INFINITY ? tc::ex2_approx(m1.x - M) : 0.f;
        const float se = m0.y * e0 + m1.y * e1;
        const float own = grp == 0 ? e0 : e1;
        const int64_t si = cur.g0 + smp;
        const bool valid = smp < cur.n;
        const float wt = sample(s0, 6);
        const bool ok = valid && se > 0.f;
        const float scale = ok ? wt * own * tc::rcp_approx(se) : 0.f;
        const float li = se > 0.f ? kLn2 * (M + tc::lg2_approx(se)) : -INFINITY;   // natural log
        if (grp == 0 && valid && loglik != nullptr) loglik[si] = li;
        wait_mma(&bar2, ph2, g2_pending);         // GEMM 2(t-1)
        if (cur.first && prev_c >= 0) flush(prev_c);   // tile t-1 closed unit prev_c
        if (grp == 0 && valid) {
            accW += wt;
            accL += wt > 0.f ? wt * li : 0.f;
        }
        // rows of this group: (h, j, kk) -> 3 KG h + KG j + kk, j = 0: w r, 1: w r g, 2: w r g^2
        {
            float a[3 * KG];
#pragma unroll
            for (int j = 0; j < KG; ++j) {
                const float wr = ok ? lk[j] * scale : 0.f;
                a[j] = wr;
                a[KG + j] = wr * gk[j];
                a[2 * KG + j] = wr * gk[j] * gk[j];
            }
#pragma unroll
            for (int b = 0; b < 3 * KG; b += 8) sts_split_bf16<8>(aA2 + b * 16, aA2 + b * 16 + P::kHalfA, a + b);
        }
        signal(&rdy2);
        a2_ready = true;
        a2_restart = cur.first;
        tc::cp_async_wait<0>();                  // tile t+2's samples, read after the barrier
        sync_pair();
        if (aborted) break;
        prev_c = cur.c;
        cur = nxt;
        nxt = nn;
        ++t;
        const int sr = s0;
        s0 = s1;
        s1 = s2;
        s2 = sr;
        b1 = b1 + 1 == P::kNB ? 0 : b1 + 1;
    }
    // ---- the last tile's GEMM 2, then its unit
    if (!aborted && a2_ready) {
        if (warp == 4) issue_g2(t - 1, a2_restart);
        g2_pending = true;
        wait_mma(&bar2, ph2, g2_pending);
        flush(prev_c);
    }
    tc::cp_async_wait<0>();
    // drain every product still in flight (after a timeout) before TMEM is freed
    if (g1_pending && !tc::mbar_wait_bounded(&bar1, ph1, kTcWaitNs) && lane == 0) atomicExch(&ws->err, 1);
    if (g2_pending && !tc::mbar_wait_bounded(&bar2, ph2, kTcWaitNs) && lane == 0) atomicExch(&ws->err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(td, P::kCols);
}

size_t tc_smem_bytes(int K, int prec) {
#define SDMM_TC_BYTES(KK, PP) \
    if (K == KK && prec == PP) return (size_t)TcPlan<KK, PP>::kBytes;
    SDMM_TC_BYTES(16, SDMM_PREC_TC_3XBF16) SDMM_TC_BYTES(16, SDMM_PREC_TC_TF32)
    SDMM_TC_BYTES(16, SDMM_PREC_TC_3XTF32) SDMM_TC_BYTES(32, SDMM_PREC_TC_3XBF16)
    SDMM_TC_BYTES(32, SDMM_PREC_TC_TF32) SDMM_TC_BYTES(32, SDMM_PREC_TC_3XTF32)
    SDMM_TC_BYTES(16, SDMM_PREC_TC_6XBF16) SDMM_TC_BYTES(32, SDMM_PREC_TC_6XBF16)
#undef SDMM_TC_BYTES
    return 0;
}

int tc_ctas_per_sm(int K, int prec) {
#define SDMM_TC_CTAS(KK, PP) \
    if (K == KK && prec == PP) return TcPlan<KK, PP>::kCtas;
    SDMM_TC_CTAS(16, SDMM_PREC_TC_3XBF16) SDMM_TC_CTAS(16, SDMM_PREC_TC_TF32)
    SDMM_TC_CTAS(16, SDMM_PREC_TC_3XTF32) SDMM_TC_CTAS(32, SDMM_PREC_TC_3XBF16)
    SDMM_TC_CTAS(32, SDMM_PREC_TC_TF32) SDMM_TC_CTAS(32, SDMM_PREC_TC_3XTF32)
    SDMM_TC_CTAS(16, SDMM_PREC_TC_6XBF16) SDMM_TC_CTAS(32, SDMM_PREC_TC_6XBF16)
#undef SDMM_TC_CTAS
    return 1;
}

cudaError_t launch_tc_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st, float* ctab,
                              float* xref, int euclid) {
    const int64_t n = R * K;
    k_tc_prepare<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(K, R, st, ctab, xref, euclid);
    return cudaGetLastError();
}

template <int K, int PREC, bool EU>
static cudaError_t launch_tc_estep_t(cudaStream_t s, int grid, WsHeader* ws, const int32_t* cr,
                                     const int64_t* units, const float* ctab, const float* xref,
                                     float* partial, int ps, int write_ll, int solid) {
    const int bytes = TcPlan<K, PREC>::kBytes;
    cudaError_t e =
        cudaFuncSetAttribute(k_tc_estep<K, PREC, EU>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    k_tc_estep<K, PREC, EU><<<grid, kTcThreads, bytes, s>>>(ws, cr, units, ctab, xref, partial, ps, write_ll,
                                                            solid);
    return cudaGetLastError();
}

cudaError_t launch_tc_estep(cudaStream_t s, int K, int prec, int grid, WsHeader* ws, const int32_t* cr,
                            const int64_t* units, const float* ctab, const float* xref, float* partial,
                            int ps, int write_ll, int euclid, int solid) {
#define SDMM_TC_CASE(KK, PP) \
    if (!euclid && K == KK && prec == PP) \
        return launch_tc_estep_t<KK, PP, false>(s, grid, ws, cr, units, ctab, xref, partial, ps, write_ll, \
                                                solid);
#define SDMM_TC_CASE_EU(KK, PP) \
    if (euclid && K == KK && prec == PP) \
        return launch_tc_estep_t<KK, PP, true>(s, grid, ws, cr, units, ctab, xref, partial, ps, write_ll, 0);
    SDMM_TC_CASE(16, SDMM_PREC_TC_3XBF16) SDMM_TC_CASE(16, SDMM_PREC_TC_TF32)
    SDMM_TC_CASE(16, SDMM_PREC_TC_3XTF32) SDMM_TC_CASE(32, SDMM_PREC_TC_3XBF16)
    SDMM_TC_CASE(32, SDMM_PREC_TC_TF32) SDMM_TC_CASE(32, SDMM_PREC_TC_3XTF32)
    SDMM_TC_CASE(16, SDMM_PREC_TC_6XBF16) SDMM_TC_CASE(32, SDMM_PREC_TC_6XBF16)
    // the Euclidean ablation: the two forms that meet the parity contract
    SDMM_TC_CASE_EU(16, SDMM_PREC_TC_6XBF16) SDMM_TC_CASE_EU(32, SDMM_PREC_TC_6XBF16)
    SDMM_TC_CASE_EU(16, SDMM_PREC_TC_3XTF32) SDMM_TC_CASE_EU(32, SDMM_PREC_TC_3XTF32)
#undef SDMM_TC_CASE
#undef SDMM_TC_CASE_EU
    return cudaErrorInvalidValue;
}

}  // namespace sdmm
