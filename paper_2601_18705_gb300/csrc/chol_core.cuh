// chol_core.cuh -- one CholeskyQR factorisation of a reduced Gram, shared by
// the per-pass kernel (k_chol) and the fused step-8 kernel (k_lside).
//
// G is symmetric (r x r, column-major, both triangles); R (upper triangular,
// column-major) satisfies R^T R = G (+ shift I).  The elimination is
// division-free: with d the pivot of step p and 2^-e its binary exponent,
// the trailing block becomes (d C_ij - C_pi C_pj) 2^-e, i.e. the Schur
// complement of the usual elimination times a known scale sigma
// (sigma_{p+1} = sigma_p d 2^-e, always in [1, 2^p)).  Only the final
// normalisation R_pj = C_pj / sqrt(sigma_p d_p) divides (once per row, all
// rows at once), which keeps the FP64 divide and square root off the
// per-pivot chain.  Both products of an update are rounded on their own (no
// fused multiply-add), so exactly repeated columns cancel to an exact zero
// pivot.
//
// detect: the first (unshifted) attempt marks columns whose residual^2 falls
// below tau |column|^2 as dependent; if there are any, S.dep marks them,
// *ndep counts them and R is not written (the caller replaces them and
// factorises again).  Otherwise a pivot below u tr(G) restarts with a shift
// (shifted CholeskyQR, *shifted = true).  Every thread of the CTA calls it.
#pragma once

#include "dlr_internal.cuh"

namespace dlr {

// 2^-e for the binary exponent e of a normal x > 0 (x 2^-e in [1, 2))
__device__ __forceinline__ double inv_pow2_exponent(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
  return __longlong_as_double((long long)(1023 - e) << 52);
}

struct CholScratch {
  double C[32 * 32];
  double sig[33], thr_dep[33], thr_fail[33], rho[32];
  int dep[32];
  int ndep;
  double tr;
  // upper-triangle entries (i, j), i <= j, ordered by i from r-1 down, so
  // that the entries a pivot step updates (i > p) form a prefix
  unsigned short tri[32 * 33 / 2];
};

// x > thr for thr >= 0, compared as integers (non-negative doubles order
// like their bit patterns; a negative x has a negative pattern)
__device__ __forceinline__ bool above(double x, double thr) {
  return __double_as_longlong(x) > __double_as_longlong(thr);
}

__device__ __forceinline__ void chol_core(const double *G, int r, bool detect_first, double u, double tau, double *R,
                                          CholScratch &S, int *ndep_out, bool *shifted_out) {
  const int t = threadIdx.x;
  double *C = S.C;
  if (t < 32) {
    const double x = warp_sum(t < r ? G[t + r * t] : 0.0);
    if (t == 0) S.tr = x;
  }
  for (int i = t; i < r; i += blockDim.x) {  // row i of the table: offset of rows r-1 .. i+1
    const int above_rows = (r - 1 - i) * (r - i) / 2;  // entries of rows > i
    for (int j = i; j < r; ++j) S.tri[above_rows + (j - i)] = (unsigned short)(i | (j << 8));
  }
  __syncthreads();
  const double tr = S.tr;
  double shift = 0.0;
  bool shifted = false, failed = false;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const bool detect = detect_first && shift == 0.0;
    for (int e = t; e < r * r; e += blockDim.x) C[e] = G[e] + ((e % r == e / r) ? shift : 0.0);
    if (t < 32) S.dep[t] = 0;
    if (t == 0) {
      S.ndep = 0;
      S.sig[0] = 1.0;
      S.thr_dep[0] = tau * G[0];
      S.thr_fail[0] = u * tr;
    }
    __syncthreads();
    failed = false;
    for (int p = 0; p < r; ++p) {
      // the same decision in every thread, on the scaled pivot
      const double d = C[p + r * p];
      const bool is_dep = detect && !above(d, S.thr_dep[p]);
      if (!is_dep && !above(d, S.thr_fail[p])) { failed = true; break; }
      const double sc = is_dep ? 1.0 : inv_pow2_exponent(d);
      if (t == 0) {  // scale and thresholds of the next step
        const double s1 = is_dep ? S.sig[p] : S.sig[p] * (d * sc);
        S.sig[p + 1] = s1;
        if (p + 1 < r) {
          S.thr_dep[p + 1] = tau * G[(p + 1) * (r + 1)] * s1;
          S.thr_fail[p + 1] = u * tr * s1;
        }
        if (is_dep) { S.dep[p] = 1; ++S.ndep; }
      }
      if (!is_dep) {
        const int na = (r - 1 - p) * (r - p) / 2;  // entries with i > p
        for (int e = t; e < na; e += blockDim.x) {
          const int i = S.tri[e] & 0xff, j = S.tri[e] >> 8;
          C[i + r * j] = __dmul_rn(__dsub_rn(__dmul_rn(d, C[i + r * j]), __dmul_rn(C[p + r * i], C[p + r * j])), sc);
        }
      }
      __syncthreads();
    }
    if (detect && S.ndep > 0) {
      *ndep_out = S.ndep;
      *shifted_out = false;
      return;
    }
    if (!failed) break;
    shift = shift == 0.0 ? u * tr : shift * 100.0;
    shifted = true;
    __syncthreads();
  }
  // R_pj = C_pj / sqrt(sigma_p C_pp)
  if (t < r) S.rho[t] = 1.0 / sqrt(S.sig[t] * C[t * (r + 1)]);
  __syncthreads();
  for (int e = t; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    R[e] = i <= j ? C[e] * S.rho[i] : 0.0;
  }
  *ndep_out = 0;
  *shifted_out = shifted;
  __syncthreads();
}

}  // namespace dlr
