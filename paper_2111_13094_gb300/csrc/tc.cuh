// tc.cuh -- inline-PTX helpers for the 5th-generation tensor cores of
// sm_103a: TMEM allocation and loads, tcgen05.mma with shared-memory operand
// descriptors, commits to mbarriers, and bounded mbarrier waits.
//
// Operand tiles live in shared memory in the K-major layout without swizzle:
// 8-row x 16-byte "core matrices" of 128 contiguous bytes; along K the core
// matrices of a row block are adjacent (leading-dimension offset 128 B), and
// consecutive 8-row blocks are `8 * C * esize` bytes apart (stride-dimension
// offset), for a tile of C elements along K.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdmm {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a K-major tile with C elements along K
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int row, int k, int C, int esize) {
    const int per = 16 / esize;
    return (uint32_t)(((row >> 3) * (C / per) + (k / per)) * 128 + (row & 7) * 16 + (k % per) * esize);
}

// byte offset of element (mn, k) of an MN-major tile with MN elements along
// the M (or N) dimension: core matrices hold 8 K-rows of 8 contiguous MN
// elements (BF16); MN blocks are 128 B apart, K blocks (MN/8)*128 B apart.
// Its descriptor takes the K-block distance as the leading-dimension offset
// and the MN-block distance (128 B) as the stride offset.
__host__ __device__ __forceinline__ uint32_t mnmajor_offset(int mn, int k, int MN) {
    return (uint32_t)(((k >> 3) * (MN >> 3) + (mn >> 3)) * 128 + (k & 7) * 16 + (mn & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and stride
// dimension byte offsets (all >> 4), descriptor version 1 at bits 46-47, no
// swizzle (layout type 0 at bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt`
// (kind::f16: 0 = F16, 1 = BF16; kind::tf32: 2 = TF32), both K-major,
// M x N tile.
__host__ __device__ __forceinline__ uint32_t instr_desc(int fmt, int M, int N, int a_mn = 0,
                                                        int b_mn = 0) {
    uint32_t d = 0;
    d |= 1u << 4;                        // D format: F32
    d |= (uint32_t)fmt << 7;             // A format
    d |= (uint32_t)fmt << 10;            // B format
    d |= (uint32_t)(a_mn & 1) << 15;     // A: 0 K-major, 1 MN-major
    d |= (uint32_t)(b_mn & 1) << 16;     // B: 0 K-major, 1 MN-major
    d |= (uint32_t)(N >> 3) << 17;       // N / 8
    d |= (uint32_t)(M >> 4) << 24;       // M / 16
    return d;
}

// ---- TMEM (one warp executes these)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(dst_smem)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols)
                 : "memory");
}

// ---- MMA issue (one thread): D[tmem] (+)= A[smem] * B[smem]^T
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
// arrive on `bar` once all MMAs issued so far by this thread have completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_addr(bar)) : "memory");
}

// ---- ordering
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// make this thread's generic-proxy shared-memory writes visible to the tensor core
__device__ __forceinline__ void fence_smem_to_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// as mbar_try_wait, but the thread may stay suspended (without issuing) for up
// to `hint_ns` nanoseconds while the phase is still incomplete
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `parity` of `bar` for at most `limit_ns` nanoseconds.
// Returns false on timeout (the caller records an error and stops).
// Each poll suspends the thread for up to 0.1 ms, so waiting costs almost no
// issue slots.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait_hint(bar, parity, 100000u)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// ---- shared memory through 32-bit shared-window addresses
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}
__device__ __forceinline__ void sts64(uint32_t a, uint32_t x, uint32_t y) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" :: "r"(a), "r"(x), "r"(y) : "memory");
}
__device__ __forceinline__ void sts32(uint32_t a, float x) {
    asm volatile("st.shared.f32 [%0], %1;" :: "r"(a), "f"(x) : "memory");
}
__device__ __forceinline__ float lds32(uint32_t a) {
    float x;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x) : "r"(a) : "memory");
    return x;
}
__device__ __forceinline__ float2 lds64(uint32_t a) {
    float2 x;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x.x), "=f"(x.y) : "r"(a) : "memory");
    return x;
}
// 4-byte asynchronous copy global -> shared (shared-window address; zero
// fill when `valid` is false, `src` must still be a readable address)
__device__ __forceinline__ void cp_async4s(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

// completion of this thread's asynchronous copies: commit / wait groups
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// arrive once on `bar` (release, CTA scope)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(bar)) : "memory");
}

// named barrier ID over N threads that returns whether any of them passed p != 0
template <int ID, int N>
__device__ __forceinline__ bool bar_red_or(bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, s;\n\tsetp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred s, %2, %3, q;\n\tselp.u32 %0, 1, 0, s;\n\t}\n"
        : "=r"(r) : "r"((uint32_t)p), "n"(ID), "n"(N) : "memory");
    return r != 0;
}

// shared-memory descriptor moved by `bytes` (the address field is the low 14
// bits of the descriptor, in 16-byte units; callers stay inside one tile)
__device__ __forceinline__ uint64_t desc_add(uint64_t d, uint32_t bytes) { return d + (uint64_t)(bytes >> 4); }

// ---- TMEM -> registers: 32 lanes x 32 bit, 16 consecutive columns per
// thread (lane quadrant of the calling warp), waiting for the load in the
// same statement so that no register is read early
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Single-instruction approximations of the special-function unit (PTX
// .approx.ftz forms; inputs and results flush subnormals to zero)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 -> TF32 (round to nearest, ties away), kept in a 32-bit container
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace sdmm
