// Inline-PTX wrappers for the Blackwell (sm_103a) features the matrixized
// kernels use: mbarriers, TMA (cp.async.bulk.tensor), bulk copies, and the
// 5th-generation tensor-core instructions (tcgen05.alloc / mma / commit / ld).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace stx {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Test the phase with the given parity; when it is not complete the thread is
// suspended in hardware until the phase completes or about a millisecond has
// passed (suspend-time hint), so waiting warps take no issue slots from the
// warps doing the work.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(0x100000u)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most
// `limit_cycles` SM clock cycles.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit_cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit_cycles) return false;
    }
    return true;
}

// ------------------------------------------------------------------ TMA / bulk copies
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Tiled shared -> global store of one box (bulk-group completion); writes
// outside the tensor are dropped.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int c0, int c1, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(map), "r"(c0),
                 "r"(c1), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit_group() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// Wait until at most N committed bulk groups of this thread still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_group_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}

// Wait until at most N committed bulk groups of this thread are incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait_group() {
    asm volatile("cp.async.bulk.wait_group %0;\n" ::"n"(N) : "memory");
}

// Named barrier over `count` threads (id 1..15; id 0 is __syncthreads).
__device__ __forceinline__ void named_barrier(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// Contiguous global -> shared copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Make generic-proxy shared-memory writes visible to the async proxy (TMA, tensor cores).
// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their memory operations are visible (a no-op for a
// grid launched without the attribute); let dependents launch early.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// ------------------------------------------------------------------ tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// D[tmem] (+)= A[tmem] x B[smem desc], FP32 accumulate; A is read from
// tensor memory (lane = row of A).  KIND_F16: BF16 (or FP16) inputs per the
// instruction descriptor, two 16-bit elements per 32-bit column (lower k in
// the low half); else TF32, one element per column.  CLEAR: D = A x B (the
// first MMA of an accumulation), else D += A x B.  The accumulate choice is
// part of the instruction text, not a run-time predicate, so a clearing MMA
// and an accumulating one are never the same asm statement with different
// operands.
template <bool KIND_F16, bool CLEAR>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc) {
    if constexpr (KIND_F16 && CLEAR)
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 0;\n" ::"r"(d_tmem), "r"(a_tmem),
                     "l"(bdesc), "r"(idesc)
                     : "memory");
    else if constexpr (KIND_F16)
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 1;\n" ::"r"(d_tmem), "r"(a_tmem),
                     "l"(bdesc), "r"(idesc)
                     : "memory");
    else if constexpr (CLEAR)
        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 0;\n" ::"r"(d_tmem), "r"(a_tmem),
                     "l"(bdesc), "r"(idesc)
                     : "memory");
    else
        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d_tmem), "r"(a_tmem),
                     "l"(bdesc), "r"(idesc)
                     : "memory");
}

// Arrive on `bar` once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Tensor-memory loads and stores complete asynchronously: tcgen05.ld writes
// its destination registers, and tcgen05.st reads its source registers, some
// time after the instruction issues, until tcgen05.wait::ld / ::st.  The
// compiler cannot see that, so if the load, the store and the wait were
// separate asm statements it could copy, spill or reuse those registers in
// between (under register pressure it does).  Every load and store here is
// therefore fused with its wait in one asm statement: the outputs are
// defined, and the inputs released, only once the transfer has completed.
//
// tmem_ld_xW_sync(a0, r0, a1, r1, ...): 32 lanes x W consecutive 32-bit
// columns from each address; thread t of the warp receives lane (base + t).
// 4 columns per block (32x32b.x4), 1-4 blocks, then the wait.
__device__ __forceinline__ void tmem_ld_x4_sync(uint32_t a0, uint32_t (&r0)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3])
        : "r"(a0)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x4_sync(uint32_t a0, uint32_t (&r0)[4], uint32_t a1, uint32_t (&r1)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%8];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%9];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3])
        : "r"(a0), "r"(a1)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x4_sync(uint32_t a0, uint32_t (&r0)[4], uint32_t a1, uint32_t (&r1)[4], uint32_t a2, uint32_t (&r2)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%13];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%14];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3])
        : "r"(a0), "r"(a1), "r"(a2)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x4_sync(uint32_t a0, uint32_t (&r0)[4], uint32_t a1, uint32_t (&r1)[4], uint32_t a2, uint32_t (&r2)[4], uint32_t a3, uint32_t (&r3)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%17];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%18];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%19];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3]), "=r"(r3[0]), "=r"(r3[1]), "=r"(r3[2]), "=r"(r3[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x8_sync(uint32_t a0, uint32_t (&r0)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7])
        : "r"(a0)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x8_sync(uint32_t a0, uint32_t (&r0)[8], uint32_t a1, uint32_t (&r1)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7])
        : "r"(a0), "r"(a1)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x8_sync(uint32_t a0, uint32_t (&r0)[8], uint32_t a1, uint32_t (&r1)[8], uint32_t a2, uint32_t (&r2)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%25];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%26];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]), "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3]), "=r"(r2[4]), "=r"(r2[5]), "=r"(r2[6]), "=r"(r2[7])
        : "r"(a0), "r"(a1), "r"(a2)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x8_sync(uint32_t a0, uint32_t (&r0)[8], uint32_t a1, uint32_t (&r1)[8], uint32_t a2, uint32_t (&r2)[8], uint32_t a3, uint32_t (&r3)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%33];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%34];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%35];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]), "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3]), "=r"(r2[4]), "=r"(r2[5]), "=r"(r2[6]), "=r"(r2[7]), "=r"(r3[0]), "=r"(r3[1]), "=r"(r3[2]), "=r"(r3[3]), "=r"(r3[4]), "=r"(r3[5]), "=r"(r3[6]), "=r"(r3[7])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x16_sync(uint32_t a0, uint32_t (&r0)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r0[8]), "=r"(r0[9]), "=r"(r0[10]), "=r"(r0[11]), "=r"(r0[12]), "=r"(r0[13]), "=r"(r0[14]), "=r"(r0[15])
        : "r"(a0)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x16_sync(uint32_t a0, uint32_t (&r0)[16], uint32_t a1, uint32_t (&r1)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r0[8]), "=r"(r0[9]), "=r"(r0[10]), "=r"(r0[11]), "=r"(r0[12]), "=r"(r0[13]), "=r"(r0[14]), "=r"(r0[15]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]), "=r"(r1[8]), "=r"(r1[9]), "=r"(r1[10]), "=r"(r1[11]), "=r"(r1[12]), "=r"(r1[13]), "=r"(r1[14]), "=r"(r1[15])
        : "r"(a0), "r"(a1)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x16_sync(uint32_t a0, uint32_t (&r0)[16], uint32_t a1, uint32_t (&r1)[16], uint32_t a2, uint32_t (&r2)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%48];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%49];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%50];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r0[8]), "=r"(r0[9]), "=r"(r0[10]), "=r"(r0[11]), "=r"(r0[12]), "=r"(r0[13]), "=r"(r0[14]), "=r"(r0[15]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]), "=r"(r1[8]), "=r"(r1[9]), "=r"(r1[10]), "=r"(r1[11]), "=r"(r1[12]), "=r"(r1[13]), "=r"(r1[14]), "=r"(r1[15]), "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3]), "=r"(r2[4]), "=r"(r2[5]), "=r"(r2[6]), "=r"(r2[7]), "=r"(r2[8]), "=r"(r2[9]), "=r"(r2[10]), "=r"(r2[11]), "=r"(r2[12]), "=r"(r2[13]), "=r"(r2[14]), "=r"(r2[15])
        : "r"(a0), "r"(a1), "r"(a2)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_x16_sync(uint32_t a0, uint32_t (&r0)[16], uint32_t a1, uint32_t (&r1)[16], uint32_t a2, uint32_t (&r2)[16], uint32_t a3, uint32_t (&r3)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%65];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%66];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%67];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]), "=r"(r0[8]), "=r"(r0[9]), "=r"(r0[10]), "=r"(r0[11]), "=r"(r0[12]), "=r"(r0[13]), "=r"(r0[14]), "=r"(r0[15]), "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]), "=r"(r1[8]), "=r"(r1[9]), "=r"(r1[10]), "=r"(r1[11]), "=r"(r1[12]), "=r"(r1[13]), "=r"(r1[14]), "=r"(r1[15]), "=r"(r2[0]), "=r"(r2[1]), "=r"(r2[2]), "=r"(r2[3]), "=r"(r2[4]), "=r"(r2[5]), "=r"(r2[6]), "=r"(r2[7]), "=r"(r2[8]), "=r"(r2[9]), "=r"(r2[10]), "=r"(r2[11]), "=r"(r2[12]), "=r"(r2[13]), "=r"(r2[14]), "=r"(r2[15]), "=r"(r3[0]), "=r"(r3[1]), "=r"(r3[2]), "=r"(r3[3]), "=r"(r3[4]), "=r"(r3[5]), "=r"(r3[6]), "=r"(r3[7]), "=r"(r3[8]), "=r"(r3[9]), "=r"(r3[10]), "=r"(r3[11]), "=r"(r3[12]), "=r"(r3[13]), "=r"(r3[14]), "=r"(r3[15])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
        : "memory");
}

// tmem_st_x8_sync(a0, v0, ...): 32 lanes x 8 consecutive 32-bit columns at
// each address; thread t of the warp writes lane (base + t).
__device__ __forceinline__ void tmem_st_x8_sync(uint32_t a0, const uint32_t (&v0)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
        "tcgen05.wait::st.sync.aligned;\n"
        :
        : "r"(a0), "r"(v0[0]), "r"(v0[1]), "r"(v0[2]), "r"(v0[3]), "r"(v0[4]), "r"(v0[5]), "r"(v0[6]), "r"(v0[7])
        : "memory");
}

__device__ __forceinline__ void tmem_st_x8_sync(uint32_t a0, const uint32_t (&v0)[8], uint32_t a1, const uint32_t (&v1)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%10, %11, %12, %13, %14, %15, %16, %17};\n"
        "tcgen05.wait::st.sync.aligned;\n"
        :
        : "r"(a0), "r"(a1), "r"(v0[0]), "r"(v0[1]), "r"(v0[2]), "r"(v0[3]), "r"(v0[4]), "r"(v0[5]), "r"(v0[6]), "r"(v0[7]), "r"(v1[0]), "r"(v1[1]), "r"(v1[2]), "r"(v1[3]), "r"(v1[4]), "r"(v1[5]), "r"(v1[6]), "r"(v1[7])
        : "memory");
}

__device__ __forceinline__ void tmem_st_x8_sync(uint32_t a0, const uint32_t (&v0)[8], uint32_t a1, const uint32_t (&v1)[8], uint32_t a2, const uint32_t (&v2)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%3, %4, %5, %6, %7, %8, %9, %10};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%11, %12, %13, %14, %15, %16, %17, %18};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%2], {%19, %20, %21, %22, %23, %24, %25, %26};\n"
        "tcgen05.wait::st.sync.aligned;\n"
        :
        : "r"(a0), "r"(a1), "r"(a2), "r"(v0[0]), "r"(v0[1]), "r"(v0[2]), "r"(v0[3]), "r"(v0[4]), "r"(v0[5]), "r"(v0[6]), "r"(v0[7]), "r"(v1[0]), "r"(v1[1]), "r"(v1[2]), "r"(v1[3]), "r"(v1[4]), "r"(v1[5]), "r"(v1[6]), "r"(v1[7]), "r"(v2[0]), "r"(v2[1]), "r"(v2[2]), "r"(v2[3]), "r"(v2[4]), "r"(v2[5]), "r"(v2[6]), "r"(v2[7])
        : "memory");
}

__device__ __forceinline__ void tmem_st_x8_sync(uint32_t a0, const uint32_t (&v0)[8], uint32_t a1, const uint32_t (&v1)[8], uint32_t a2, const uint32_t (&v2)[8], uint32_t a3, const uint32_t (&v3)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%4, %5, %6, %7, %8, %9, %10, %11};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%12, %13, %14, %15, %16, %17, %18, %19};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%2], {%20, %21, %22, %23, %24, %25, %26, %27};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%3], {%28, %29, %30, %31, %32, %33, %34, %35};\n"
        "tcgen05.wait::st.sync.aligned;\n"
        :
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(v0[0]), "r"(v0[1]), "r"(v0[2]), "r"(v0[3]), "r"(v0[4]), "r"(v0[5]), "r"(v0[6]), "r"(v0[7]), "r"(v1[0]), "r"(v1[1]), "r"(v1[2]), "r"(v1[3]), "r"(v1[4]), "r"(v1[5]), "r"(v1[6]), "r"(v1[7]), "r"(v2[0]), "r"(v2[1]), "r"(v2[2]), "r"(v2[3]), "r"(v2[4]), "r"(v2[5]), "r"(v2[6]), "r"(v2[7]), "r"(v3[0]), "r"(v3[1]), "r"(v3[2]), "r"(v3[3]), "r"(v3[4]), "r"(v3[5]), "r"(v3[6]), "r"(v3[7])
        : "memory");
}

__device__ __forceinline__ void tmem_st_x8_sync(uint32_t a0, const uint32_t (&v0)[8], uint32_t a1, const uint32_t (&v1)[8], uint32_t a2, const uint32_t (&v2)[8], uint32_t a3, const uint32_t (&v3)[8], uint32_t a4, const uint32_t (&v4)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%5, %6, %7, %8, %9, %10, %11, %12};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%13, %14, %15, %16, %17, %18, %19, %20};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%2], {%21, %22, %23, %24, %25, %26, %27, %28};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%3], {%29, %30, %31, %32, %33, %34, %35, %36};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%4], {%37, %38, %39, %40, %41, %42, %43, %44};\n"
        "tcgen05.wait::st.sync.aligned;\n"
        :
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(v0[0]), "r"(v0[1]), "r"(v0[2]), "r"(v0[3]), "r"(v0[4]), "r"(v0[5]), "r"(v0[6]), "r"(v0[7]), "r"(v1[0]), "r"(v1[1]), "r"(v1[2]), "r"(v1[3]), "r"(v1[4]), "r"(v1[5]), "r"(v1[6]), "r"(v1[7]), "r"(v2[0]), "r"(v2[1]), "r"(v2[2]), "r"(v2[3]), "r"(v2[4]), "r"(v2[5]), "r"(v2[6]), "r"(v2[7]), "r"(v3[0]), "r"(v3[1]), "r"(v3[2]), "r"(v3[3]), "r"(v3[4]), "r"(v3[5]), "r"(v3[6]), "r"(v3[7]), "r"(v4[0]), "r"(v4[1]), "r"(v4[2]), "r"(v4[3]), "r"(v4[4]), "r"(v4[5]), "r"(v4[6]), "r"(v4[7])
        : "memory");
}

__device__ __forceinline__ void tmem_st_x8_sync(uint32_t a0, const uint32_t (&v0)[8], uint32_t a1, const uint32_t (&v1)[8], uint32_t a2, const uint32_t (&v2)[8], uint32_t a3, const uint32_t (&v3)[8], uint32_t a4, const uint32_t (&v4)[8], uint32_t a5, const uint32_t (&v5)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%6, %7, %8, %9, %10, %11, %12, %13};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%14, %15, %16, %17, %18, %19, %20, %21};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%2], {%22, %23, %24, %25, %26, %27, %28, %29};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%3], {%30, %31, %32, %33, %34, %35, %36, %37};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%4], {%38, %39, %40, %41, %42, %43, %44, %45};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%5], {%46, %47, %48, %49, %50, %51, %52, %53};\n"
        "tcgen05.wait::st.sync.aligned;\n"
        :
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(v0[0]), "r"(v0[1]), "r"(v0[2]), "r"(v0[3]), "r"(v0[4]), "r"(v0[5]), "r"(v0[6]), "r"(v0[7]), "r"(v1[0]), "r"(v1[1]), "r"(v1[2]), "r"(v1[3]), "r"(v1[4]), "r"(v1[5]), "r"(v1[6]), "r"(v1[7]), "r"(v2[0]), "r"(v2[1]), "r"(v2[2]), "r"(v2[3]), "r"(v2[4]), "r"(v2[5]), "r"(v2[6]), "r"(v2[7]), "r"(v3[0]), "r"(v3[1]), "r"(v3[2]), "r"(v3[3]), "r"(v3[4]), "r"(v3[5]), "r"(v3[6]), "r"(v3[7]), "r"(v4[0]), "r"(v4[1]), "r"(v4[2]), "r"(v4[3]), "r"(v4[4]), "r"(v4[5]), "r"(v4[6]), "r"(v4[7]), "r"(v5[0]), "r"(v5[1]), "r"(v5[2]), "r"(v5[3]), "r"(v5[4]), "r"(v5[5]), "r"(v5[6]), "r"(v5[7])
        : "memory");
}

// tmem_st_x8_sync over an array of S stores (compile-time S = 1..6): one asm
// statement, one wait.
template <int S>
__device__ __forceinline__ void tmem_st_x8_sync_n(const uint32_t (&a)[S], const uint32_t (&v)[S][8]) {
    static_assert(S >= 1 && S <= 6, "1..6 stores");
    if constexpr (S == 1) tmem_st_x8_sync(a[0], v[0]);
    if constexpr (S == 2) tmem_st_x8_sync(a[0], v[0], a[1], v[1]);
    if constexpr (S == 3) tmem_st_x8_sync(a[0], v[0], a[1], v[1], a[2], v[2]);
    if constexpr (S == 4) tmem_st_x8_sync(a[0], v[0], a[1], v[1], a[2], v[2], a[3], v[3]);
    if constexpr (S == 5) tmem_st_x8_sync(a[0], v[0], a[1], v[1], a[2], v[2], a[3], v[3], a[4], v[4]);
    if constexpr (S == 6) tmem_st_x8_sync(a[0], v[0], a[1], v[1], a[2], v[2], a[3], v[3], a[4], v[4], a[5], v[5]);
}

// Shared-memory matrix descriptor, no swizzle (canonical K-major layout of
// 8-row x 16-byte core matrices): start address, LBO = byte distance between
// core matrices adjacent along K, SBO = byte distance between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, relative LBO, swizzle mode 0 (none)
}

// Instruction descriptor (kind::tf32 / kind::f16): FP32 accumulator, both
// operands K-major, dense.  a_fmt/b_fmt: 0 = F16, 1 = BF16, 2 = TF32.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t a_fmt, uint32_t b_fmt, uint32_t m, uint32_t n) {
    return (1u << 4) | (a_fmt << 7) | (b_fmt << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest, ties away.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace ptx
}  // namespace stx
