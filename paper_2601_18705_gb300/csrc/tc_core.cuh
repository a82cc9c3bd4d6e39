// tc_core.cuh -- the fifth-generation tensor cores (tcgen05) for TF32
// contractions: D (FP32, in tensor memory) += A B^T with A (M x K) and
// B (N x K) in shared memory, both K-major without swizzle (the projections
// k_project_tc5 in k_dense.cu, and dlr_debug_tc_gemm in k_tcgemm.cu).
//
// Operand layout.  An operand tile of R rows and 8 TF32 columns (one
// k-step of an MMA) is made of core matrices of 8 rows x 16 bytes (4 TF32
// values of a row, contiguous; row i of a core matrix at +16 i bytes).  In
// this project a tile keeps the two core matrices of 8 rows side by side
// (the K-adjacent one at +128 bytes, the descriptor's leading byte offset)
// and consecutive 8-row groups 256 bytes apart (the stride byte offset), so
// a tile is R x 32 bytes; tiles of consecutive k-steps follow each other.
//
// Split TF32 products.  A value x is stored as hi = x rounded to TF32 and
// lo = x - hi (exact in FP32; the tensor core reads its TF32 part), in two
// operand copies, and a product is summed as hi lo + lo hi + hi hi (three
// MMAs): within about 2^-20 of the exact product, of either sign.
//
// Every wait on a tensor-core completion is bounded in time.
#pragma once
#include <cstdint>

namespace dlr {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row i, column j) of an operand of R rows (any
// multiple of 8) whose tiles of 8 columns follow each other.
__host__ __device__ __forceinline__ uint32_t op_offset(int R, int i, int j) {
  return (uint32_t)((j >> 3) * (R * 32) + (i >> 3) * 256 + ((j >> 2) & 1) * 128 + (i & 7) * 16 + (j & 3) * 4);
}

// Shared-memory matrix descriptor: start address, leading byte offset (K
// direction, 128), stride byte offset (8-row groups, 256), all in 16-byte
// units; descriptor version 1 (bits 46-47), no swizzle (layout type 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t start) {
  return (uint64_t)((start >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B in
// TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// d_tmem (+)= A B^T for one k-step (issued by one thread).
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// The mbarrier receives one arrival once every MMA this thread issued so
// far has completed.
__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
               : "memory");
}

// Tensor-memory allocation by one whole warp: the base address is written
// to *slot (shared memory).
__device__ __forceinline__ void alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// this thread's generic shared-memory writes become visible to the tensor
// core (the async proxy)
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(m)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  fence_smem_to_async();
}
__device__ __forceinline__ bool mbar_test(uint64_t *m, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of the given parity (true: it completed).
__device__ __forceinline__ bool mbar_wait(uint64_t *m, unsigned parity, uint64_t limit_ns) {
  if (mbar_test(m, parity)) return true;
  const uint64_t t0 = now_ns();
  for (unsigned spins = 1;; ++spins) {
    if (mbar_test(m, parity)) return true;
    if ((spins & 63u) == 0 && now_ns() - t0 > limit_ns) return false;
  }
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane (a warp
// reads lanes 32 (warp % 4) .. + 31; taddr carries the lane in bits 16-31).
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo: hi = x rounded to TF32 (to nearest, ties away from zero, by
// integer arithmetic on the bits of a finite x), lo = x - hi exactly.
__device__ __forceinline__ void split(float x, float &hi, float &lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
  lo = x - hi;
}

}  // namespace tc
}  // namespace dlr
