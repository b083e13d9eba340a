// tc_fit.cu -- tensor-core (tcgen05) kernels.
//
//  k_tc_selftest   D = A B^T for one 128-row tile through the same shared-
//                  memory layout, descriptors, MMA issue, commit and TMEM
//                  read-out helpers that the contraction-form E-step uses.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace sdmm {

constexpr uint64_t kTcWaitNs = 2000000000ull;   // 2 s bound on any MMA wait

__global__ void __launch_bounds__(128) k_tc_selftest(int kind, int N, int Kd, const float* __restrict__ A,
                                                     const float* __restrict__ B, float* __restrict__ D,
                                                     int variant, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int esize = kind == 0 ? 2 : 4;
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * Kd * esize;
    for (int e = tid; e < 128 * Kd; e += 128) {
        const int row = e / Kd, k = e % Kd;
        const uint32_t o = tc::kmajor_offset(row, k, Kd, esize);
        if (kind == 0) *reinterpret_cast<__nv_bfloat16*>(sA + o) = __float2bfloat16_rn(A[e]);
        else *reinterpret_cast<float*>(sA + o) = tc::to_tf32(A[e]);
    }
    for (int e = tid; e < N * Kd; e += 128) {
        const int row = e / Kd, k = e % Kd;
        const uint32_t o = tc::kmajor_offset(row, k, Kd, esize);
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
        const uint32_t lbo_k = 128, sbo_m = 8u * Kd * esize;
        const uint32_t lbo = variant == 0 ? lbo_k : sbo_m;
        const uint32_t sbo = variant == 0 ? sbo_m : lbo_k;
        const int kstep = kind == 0 ? 16 : 8;
        const uint32_t idesc = tc::instr_desc(kind == 0 ? 1 : 2, 128, N);
        for (int s = 0; s < Kd / kstep; ++s) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + s * 256, lbo, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + s * 256, lbo, sbo);
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
    const int esize = kind == 0 ? 2 : 4;
    const size_t smem = (size_t)(128 + N) * Kd * esize;
    cudaError_t e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_selftest<<<1, 128, smem, s>>>(kind, N, Kd, A, B, D, variant, status);
    return cudaGetLastError();
}

}  // namespace sdmm
