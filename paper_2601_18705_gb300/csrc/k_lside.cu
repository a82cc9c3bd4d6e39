// k_lside.cu -- step 8 of Algorithm 1 (L = S W^T) in one thread-block
// cluster per instance, for the pivoted-QR angle choice (S kept general,
// U = V = I between steps).  The rows of M = diag(sqrt w) L^T are spread over
// the shared memory of the cluster's CTAs and stay there for the whole
// CholeskyQR2 (a third pass when a pass needed a shift, and orthonormal
// completion of dependent columns): each Gram is summed over the cluster
// through distributed shared memory (the same fixed order in every CTA, so
// every CTA holds the same Gram and factorises it itself), and
// Q = M R^-1 is applied in place by forward substitution.  Then S = M^T Q,
// W0 = diag(1/sqrt w) Q and vphi = L w.  This replaces the chain of Gram,
// Cholesky, completion and apply kernels (and their round trips through
// global memory) for K up to kLsideMaxK angles.
#include "chol_core.cuh"
#include "dlr_internal.cuh"

namespace dlr {

// Step 8 runs in one cluster for up to this many angles.  The cluster's FP64
// work grows with the angles while it holds 8 SMs: at 2048 angles and rank
// 32 it took 0.56 ms against 0.38 ms for the chain of kernels spread over
// the whole GPU (lognormal1024, mixed), at 1024 and below it is the faster.
constexpr int kLsideMaxK = 1024;
int lside_max_k() { return kLsideMaxK; }

// out[e] = sum over the cluster's CTAs (rank order) of part[e], e < n, in
// every CTA
__device__ __forceinline__ void cluster_allreduce(cg::cluster_group &cl, double *part, double *out, int n) {
  cl.sync();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kCl; ++q) s += cl.map_shared_rank(part, q)[e];
    out[e] = s;
  }
  cl.sync();  // no CTA refills part before every read is done
}

// local Gram of rows [0, ns) of A (rows of r): part = A^T B (both triangles
// for a symmetric one, A == B)
__device__ __forceinline__ void local_gram(const double *A, const double *B, int ns, int r, bool sym,
                                           double *part) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    if (sym && i > j) continue;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int c = 0;
    for (; c + 4 <= ns; c += 4) {
      s0 += A[c * r + i] * B[c * r + j];
      s1 += A[(c + 1) * r + i] * B[(c + 1) * r + j];
      s2 += A[(c + 2) * r + i] * B[(c + 2) * r + j];
      s3 += A[(c + 3) * r + i] * B[(c + 3) * r + j];
    }
    for (; c < ns; ++c) s0 += A[c * r + i] * B[c * r + j];
    const double s = (s0 + s1) + (s2 + s3);
    part[i + r * j] = s;
    if (sym) part[j + r * i] = s;
  }
}

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(256)
k_lside(const Inst *__restrict__ insts, int slice_max) {
  pdl_wait();
  pdl_trigger();
  cg::cluster_group cl = cg::this_cluster();
  const int g = (int)cl.block_rank();
  const Inst &I = insts[blockIdx.x / kCl];
  // nothing writes the status during this kernel, so every CTA of a cluster
  // takes the same branch
  if (*I.status != kOk) return;
  const int r = I.r, K = I.K, t = threadIdx.x, lane = t & 31;
  const int slice = (K + kCl - 1) / kCl, k0 = min(K, g * slice), ns = min(K, k0 + slice) - k0;
  extern __shared__ double sh[];
  double *M = sh;                   // slice_max x r: rows of sqrt(w_k) L_k
  double *Q = M + slice_max * r;    // the factor being orthonormalised
  double *sw = Q + slice_max * r;   // sqrt(w_k)
  __shared__ double part[32 * 32 + 32], G[32 * 32 + 32], R[32 * 32], dg[32];
  __shared__ CholScratch cs;
  const double u = chol_u(I.precision == 1), tau = chol_tau(I.precision == 1);
  for (int c = t; c < ns; c += blockDim.x) sw[c] = sqrt(I.w[k0 + c]);
  __syncthreads();
  for (int e = t; e < ns * r; e += blockDim.x) {
    const int c = e / r, i = e - c * r;
    const double v = sw[c] * I.L[(size_t)r * (k0 + c) + i];
    M[e] = v;
    Q[e] = v;
  }
  __syncthreads();
  // forward substitution teams: T threads per row (a power of two <= 32),
  // enough to give the four schedulers a warp each; a thread updates every
  // T-th column, so each FP64 instruction has all its lanes busy
  int T = 1;
  while (T < 32 && 2 * T * max(ns, 1) <= 128) T *= 2;
  const int m = t & (T - 1), rows_per_pass = blockDim.x / T;
  bool shifted_any = false;
  for (int pass = 1; pass <= 3; ++pass) {
    if (pass == 3 && !shifted_any) break;
    bool detect = pass == 1;
    for (int attempt = 0; attempt < 2; ++attempt) {
      local_gram(Q, Q, ns, r, true, part);
      cluster_allreduce(cl, part, G, r * r);
      int ndep;
      bool sh;
      chol_core(G, r, detect, u, tau, R, cs, &ndep, &sh);
      if (ndep == 0) {
        shifted_any |= sh;
        break;
      }
      // orthonormal completion: dependent columns -> pseudo-random ones
      for (int e = t; e < ns * r; e += blockDim.x) {
        const int c = e / r, j = e - c * r;
        if (cs.dep[j]) Q[e] = hash_uniform(((unsigned long long)j << 40) ^ (unsigned long long)(k0 + c));
      }
      __syncthreads();
      detect = false;
    }
    // Q <- Q R^-1: x R = q row by row, column-oriented within a team
    if (t < r) dg[t] = 1.0 / R[t * (r + 1)];
    __syncthreads();
    for (int q0 = 0; q0 < ns; q0 += rows_per_pass) {
      const int q = q0 + t / T;
      const bool own = q < ns;
      double *row = Q + (size_t)(own ? q : 0) * r;
      for (int j = 0; j < r; ++j) {
        double x = 0.0;
        if (own && m == (j & (T - 1))) {
          x = row[j] * dg[j];
          row[j] = x;
        }
        x = __shfl_sync(0xffffffffu, x, (lane & ~(T - 1)) + (j & (T - 1)));
        if (own)
          for (int k = j + 1 + ((m - j - 1) & (T - 1)); k < r; k += T) row[k] -= x * R[j + r * k];
      }
    }
    __syncthreads();
  }
  // S = M^T Q and the local share of vphi = L w (w_k L_k = sqrt(w_k) M_k)
  local_gram(M, Q, ns, r, false, part);
  for (int i = t; i < r; i += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < ns; ++c) s += sw[c] * M[c * r + i];
    part[r * r + i] = s;
  }
  cluster_allreduce(cl, part, G, r * r + r);
  if (g == 0) {
    double *U = I.small + I.lay.U, *V = I.small + I.lay.V;
    for (int e = t; e < r * r; e += blockDim.x) {
      I.S0[e] = G[e];
      const double d = (e % r == e / r) ? 1.0 : 0.0;
      U[e] = d;
      V[e] = d;
    }
    for (int i = t; i < r; i += blockDim.x) I.small[I.lay.vphi + i] = G[r * r + i];
  }
  for (int e = t; e < ns * r; e += blockDim.x) {
    const int c = e / r, j = e - c * r;
    I.W0[(size_t)(k0 + c) + (size_t)K * j] = Q[e] / sw[c];
  }
}

size_t lside_smem_bytes(int slice_max, int rmax) {
  return (size_t)(2 * slice_max * rmax + slice_max) * sizeof(double);
}

cudaError_t prepare_lside(int slice_max, int rmax) {
  return cudaFuncSetAttribute(k_lside, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)lside_smem_bytes(slice_max, rmax));
}

cudaError_t launch_lside(const Inst *d, int n, int slice_max, int rmax, cudaStream_t st) {
  return launch_pdl(k_lside, dim3(n * kCl), dim3(256), lside_smem_bytes(slice_max, rmax), st, d, slice_max);
}

}  // namespace dlr
