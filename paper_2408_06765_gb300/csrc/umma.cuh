// umma.cuh -- encoders for the 5th-generation tensor-core (tcgen05) MMA of
// sm_100-family GPUs, and thin wrappers around the tcgen05 / fence PTX.
//
// Shared-memory matrix descriptor (64 bits), no-swizzle K-major layout made
// of "core matrices" of 8 rows x 16 bytes (8 x 8 bf16, rows 16 B apart):
//   bits  0-13  start address >> 4
//   bits 16-29  leading-dimension byte offset >> 4: distance between core
//               matrices adjacent along K
//   bits 32-45  stride-dimension byte offset >> 4: distance between core
//               matrices adjacent along M (or N)
//   bits 46-47  descriptor version, 1
//   bits 49-51  base offset (0), bit 52 offset mode (0 = relative)
//   bits 61-63  swizzle mode (0 = none, 2 = 128-byte)
// Instruction descriptor (32 bits) of kind::f16:
//   bits 4-5 D format (1 = f32), 7-9 A format (1 = bf16), 10-12 B format
//   (1 = bf16), 15 / 16 A / B major (0 = K-major, 1 = MN-major), 17-22 N >> 3,
//   24-28 M >> 4; everything else 0 (dense, no negation, no saturation).
#pragma once

#include <stdint.h>

namespace rsi_umma {

__host__ __device__ constexpr uint64_t smem_desc(uint32_t smem_addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return (uint64_t((smem_addr >> 4) & 0x3FFFu)) | (uint64_t((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo_bytes >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// K-major tile written by TMA with the 128-byte swizzle: rows of 64 bf16
// (128 B), atoms of 8 rows (1024 B, the stride between 8-row groups); the
// tile base is 1024-byte aligned, and the k-th 16-wide slice of K starts
// 32 k bytes into the atom (the swizzle is applied to the absolute address).
// The leading-dimension offset is unused by this layout (encoded as 1).
__host__ __device__ constexpr uint64_t smem_desc_sw128(uint32_t smem_addr) {
    return (uint64_t((smem_addr >> 4) & 0x3FFFu)) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// MN-major tile written by TMA with the 128-byte swizzle in boxes of 64 MN
// elements (128 B) x 64 k rows (8 KB, rows k at 128 B): the stride between
// 8-row groups along K is 1024 B, the stride between 64-element blocks along
// M (or N) is lbo_bytes (8 KB, one box); the k-th 16-deep slice starts
// 16 x 128 bytes further.
__host__ __device__ constexpr uint64_t smem_desc_mn_sw128(uint32_t smem_addr, uint32_t lbo_bytes) {
    return (uint64_t((smem_addr >> 4) & 0x3FFFu)) | (uint64_t((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           (uint64_t(1024 >> 4) << 32) | (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// byte offset of element (row r, k) in a K-major no-swizzle tile whose core
// matrices are LBO = 128 bytes apart along K and SBO bytes apart along rows
__host__ __device__ constexpr uint32_t core_offset(uint32_t r, uint32_t k, uint32_t sbo_bytes) {
    return (r >> 3) * sbo_bytes + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

#ifdef __CUDACC__
// 2-D tiled TMA load of box (x = inner coordinate, y = row) into shared
// memory, completing `bytes` of transaction count on mbarrier `mbar`
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int32_t x, int32_t y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}
// 2-D tiled TMA store of a shared-memory box to global memory (bulk group)
__device__ __forceinline__ void tma_store_2d(const void* tmap, int32_t x, int32_t y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap), "r"(x),
                 "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A[smem] B[smem]^T, M x N x 16, issued by one thread
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive (once) on an mbarrier when this thread's earlier tcgen05 ops are done
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp gets lane
// (warp's lane base + t), columns col .. col + 31
__device__ __forceinline__ void ld_32x32b_x32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
#endif

}  // namespace rsi_umma
