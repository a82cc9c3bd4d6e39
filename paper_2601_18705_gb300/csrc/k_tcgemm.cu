// k_tcgemm.cu -- dlr_debug_tc_gemm: the tcgen05 TF32 contraction that the
// mixed-precision projections of steps 6 and 7 (k_project_tc5) are built
// on (split TF32 products, operands in shared memory, the FP32 accumulator
// in tensor memory; tc_core.cuh), on plain device arrays, so that a test
// can check the operand layout, the descriptors and the split products
// against a reference.
#include <cuda_runtime.h>

#include "../../include/dlr.h"
#include "dlr_internal.cuh"
#include "tc_core.cuh"

namespace dlr {
int record_error(int code, const char *msg);  // message for dlr_last_error()
}

namespace {

constexpr int kTK = 32;                       // K per staged chunk (4 k-steps of 8)
constexpr uint64_t kTcWaitNs = 1000000000ull;  // bound of a completion wait

__device__ int g_tc_timed_out;

int err(int code, const char *m) { return dlr::record_error(code, m); }

size_t tc_gemm_smem(int m, int n) { return (size_t)(2 * m + 2 * n) * kTK * 4 + 16; }

// D (m x n, row-major) = A (m x k, row-major) B^T (B: n x k, row-major);
// m in {128, 256} (one or two M = 128 accumulators), n in {16, 32}, k a
// multiple of 32.  One CTA of 128 threads.
__global__ void __launch_bounds__(128) k_tc_gemm(const float *__restrict__ A, const float *__restrict__ B, int m,
                                                 int n, int k, float *__restrict__ D) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *Ah = sm, *Al = Ah + (size_t)m * kTK * 4, *Bh = Al + (size_t)m * kTK * 4;
  unsigned char *Bl = Bh + (size_t)n * kTK * 4;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(Bl + (size_t)n * kTK * 4);
  __shared__ uint32_t slot;
  __shared__ int bad;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int halves = m / 128;
  const uint32_t ncols = halves * n <= 32 ? 32u : 64u;
  if (t == 0) {
    dlr::tc::mbar_init(mbar, 1);
    bad = 0;
  }
  if (w == 0) dlr::tc::alloc(&slot, ncols);
  dlr::tc::fence_before_sync();
  __syncthreads();
  dlr::tc::fence_after_sync();
  const uint32_t tmem = slot;
  const uint32_t idesc = dlr::tc::idesc_tf32(128, n);
  unsigned parity = 0;
  for (int k0 = 0; k0 < k; k0 += kTK) {
    // this chunk's operands, split into their TF32 parts
    for (int e = t; e < (m + n) * (kTK / 4); e += blockDim.x) {
      const bool isA = e < m * (kTK / 4);
      const int ee = isA ? e : e - m * (kTK / 4);
      const int i = ee / (kTK / 4), j = 4 * (ee % (kTK / 4));
      const float4 x = *reinterpret_cast<const float4 *>((isA ? A : B) + (size_t)i * k + k0 + j);
      float4 h, l;
      dlr::tc::split(x.x, h.x, l.x);
      dlr::tc::split(x.y, h.y, l.y);
      dlr::tc::split(x.z, h.z, l.z);
      dlr::tc::split(x.w, h.w, l.w);
      const uint32_t off = dlr::tc::op_offset(isA ? m : n, i, j);
      *reinterpret_cast<float4 *>((isA ? Ah : Bh) + off) = h;
      *reinterpret_cast<float4 *>((isA ? Al : Bl) + off) = l;
    }
    dlr::tc::fence_smem_to_async();
    __syncthreads();
    if (t == 0) {
      dlr::tc::fence_after_sync();
      for (int s = 0; s < kTK / 8; ++s)
        for (int hf = 0; hf < halves; ++hf) {
          const uint32_t d = tmem + (uint32_t)(hf * n);
          const uint32_t ao = (uint32_t)(s * m * 32 + hf * 4096), bo = (uint32_t)(s * n * 32);
          const bool first = k0 == 0 && s == 0;
          dlr::tc::mma(d, dlr::tc::smem_desc(dlr::tc::saddr(Ah + ao)), dlr::tc::smem_desc(dlr::tc::saddr(Bl + bo)), idesc, !first);
          dlr::tc::mma(d, dlr::tc::smem_desc(dlr::tc::saddr(Al + ao)), dlr::tc::smem_desc(dlr::tc::saddr(Bh + bo)), idesc, true);
          dlr::tc::mma(d, dlr::tc::smem_desc(dlr::tc::saddr(Ah + ao)), dlr::tc::smem_desc(dlr::tc::saddr(Bh + bo)), idesc, true);
        }
      dlr::tc::commit(mbar);
    }
    // the operands are refilled only after the products that read them
    if (!dlr::tc::mbar_wait(mbar, parity, kTcWaitNs)) bad = 1;
    parity ^= 1u;
    __syncthreads();
    if (bad) break;
  }
  dlr::tc::fence_after_sync();
  if (!bad) {
    for (int hf = 0; hf < halves; ++hf) {
      if (w < 4) {
        const int row = 128 * hf + 32 * w + lane;
        const uint32_t ta = tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)(hf * n);
        if (n == 32) {
          float v[32];
          dlr::tc::ld32(ta, v);
#pragma unroll
          for (int c = 0; c < 32; ++c) D[(size_t)row * n + c] = v[c];
        } else {
          float v[16];
          dlr::tc::ld16(ta, v);
#pragma unroll
          for (int c = 0; c < 16; ++c) D[(size_t)row * n + c] = v[c];
        }
      }
    }
  } else if (t == 0) {
    g_tc_timed_out = 1;
  }
  dlr::tc::fence_before_sync();
  __syncthreads();
  if (w == 0) dlr::tc::dealloc(tmem, ncols);
}

}  // namespace

extern "C" int dlr_debug_tc_gemm(const float *A, const float *B, int32_t m, int32_t n, int32_t k, float *D,
                                 void *stream) {
  if (!A || !B || !D || (m != 128 && m != 256) || (n != 16 && n != 32) || k < kTK || k % kTK ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return err(DLR_EINVAL, "dlr_debug_tc_gemm: m in {128, 256}, n in {16, 32}, k a multiple of 32, "
                           "A and B 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *flag = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void **>(&flag), g_tc_timed_out) != cudaSuccess)
    return err(DLR_ECUDA, "dlr_debug_tc_gemm: symbol lookup failed");
  const size_t smem = tc_gemm_smem(m, n);
  if (cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess)
    return err(DLR_ECUDA, "dlr_debug_tc_gemm: set-up failed");
  k_tc_gemm<<<1, 128, smem, st>>>(A, B, m, n, k, D);
  int timed_out = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&timed_out, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(DLR_ECUDA, cudaGetErrorString(e));
  if (timed_out) return err(DLR_ETIMEOUT, "dlr_debug_tc_gemm: a tensor-core completion wait ran out");
  return DLR_OK;
}
