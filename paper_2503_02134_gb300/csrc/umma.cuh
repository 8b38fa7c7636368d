// tcgen05 (fifth-generation tensor core) building blocks for the BF16 GEMM
// of the learned guess's network: K-major BF16 operands staged by the
// threads into shared memory in the 128-byte-swizzled canonical layout,
// one elected thread issuing tcgen05.mma with the FP32 accumulator in
// tensor memory (TMEM), completion through tcgen05.commit on an mbarrier
// (bounded waits), and the accumulator read back with tcgen05.ld.
//
// 128-byte-swizzled K-major layout of a [R x 64] BF16 tile: row r (64
// values, 128 bytes) at byte 128 r, its 16-byte chunk c stored at chunk
// position c ^ (r mod 8) -- the XOR the hardware applies to address bits
// 4-6 from bits 7-9, so the tile base must be 1024-byte aligned.  Groups
// of 8 rows are 1024 bytes apart (the descriptor's stride-dimension byte
// offset).  One MMA consumes K = 16 (32 bytes of each row): the descriptor
// of k-step s starts 32 s bytes after the tile base.
#pragma once

#include <cuda_bf16.h>

#include "tma.cuh"

namespace sem {

constexpr int kUM = 128, kUN = 128, kUK = 64;    // CTA tile (M x N) and K per stage
constexpr int kUStages = 4;
constexpr uint32_t kUTileA = kUM * kUK * 2;      // bytes of one stage of A (16 KB)
constexpr uint32_t kUTileB = kUN * kUK * 2;      // and of B
constexpr uint32_t kUCols = kUN;                 // TMEM columns of the FP32 accumulator
constexpr size_t kUSmem = kUStages * (kUTileA + kUTileB) + 64 + 1024;   // + barriers, slot, alignment

// byte offset of 16-byte chunk c (values 8c .. 8c + 7) of row r in a
// [R x 64] K-major 128-byte-swizzled tile
__host__ __device__ constexpr uint32_t umma_chunk_off(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// shared-memory matrix descriptor: start address in 16-byte units, leading
// byte offset 1 (unused by swizzled K-major layouts), stride byte offset
// 1024 bytes (8-row groups), descriptor version 1 (bits 46-47), base offset
// 0, 128-byte swizzle (layout type 2 at bits 61-63)
__host__ __device__ constexpr uint64_t umma_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N / 8 at bits 17-22, M / 16 at bits 24-28
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// 16-byte asynchronous global -> shared copy; src_bytes 0 fills zeros (the
// source address must still be valid)
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst_smem)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D (TMEM) = A B (+ D when accum != 0), M x N x 16, issued by one thread
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// one arrive on the mbarrier once every MMA this thread issued has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane (warp w of the
// warpgroup reads lanes 32 w .. 32 w + 31), with the wait in the same block
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace sem
