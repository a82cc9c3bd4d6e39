// k_small.cu -- FP64 small dense linear algebra of the SN-like DLR step
// (Algorithm 1 of Haut et al.):
//   k_select       step 2: angle choice (column-pivoted Householder QR of W0^T,
//                  or the greedy DEIM of Section 4.2) by one thread-block
//                  cluster per instance, What, beta, gamma = What^{-T} beta,
//                  C0 = S0 What^T
//   k_chol         Cholesky of a reduced Gram (one CholeskyQR pass of steps 5
//                  and 8); detects dependent columns, shifts when needed
//   k_proj_post    step 7 Galerkin operators from the reduced projections
//   k_lstep_angle  step 7 per angle: B_k = |ox| A_x + |oy| A_y + M_t,
//                  Gauss-Jordan with partial pivoting on [B_k | I] (one warp
//                  per angle, one lane per column), B_k^{-1} kept, y_k =
//                  B_k^{-1} Q_k, both summed with weights w_k (the C-bar
//                  device of Section 3.3)
//   k_lstep_mid    (I - Cbar M_s / 4pi) Lbar = zeta
//   k_lstep_back   L_k = y_k + B_k^{-1} M_s Lbar / 4pi
//   k_svd          step 8: S = M^T Q, one-sided Jacobi SVD S = U Sigma V^T
//   k_sign         sign of each W column: its largest-magnitude entry > 0
#include "chol_core.cuh"
#include "dlr_internal.cuh"

namespace dlr {

constexpr unsigned kFullMask = 0xffffffffu;

// |x| as an integer that orders like |x| (non-negative doubles order like
// their bit patterns); integer compares stay off the FP64 pipe.
__device__ __forceinline__ long long abs_bits(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffll;
}


// ------------------------------------------------------------------
// Solve M x = b (n x n, column-major, n <= 32, in shared memory) by Gaussian
// elimination with partial pivoting, all threads of the CTA; M and b are
// overwritten, x is left in b.  The pivot is the largest magnitude in the
// column (lowest row on exact ties).  The elimination is division-free
// (rows below the pivot become (d a_ij - a_ip a_pj) 2^-e, a uniform scale
// per row), so the FP64 divides happen once per row in the back
// substitution, all at once.  Returns false (in every thread) if a pivot is
// exactly zero.
// ------------------------------------------------------------------
__device__ bool block_solve(double *M, double *b, int n) {
  __shared__ int piv_s;
  __shared__ double rdiag[32];
  const int t = threadIdx.x, lane = t & 31;
  for (int p = 0; p < n; ++p) {
    if (t < 32) {  // warp 0: pivot row (lanes = rows), integer compares of |a|
      long long v = (lane >= p && lane < n) ? abs_bits(M[lane + n * p]) : -1;
      int row = lane;
      for (int o = 16; o > 0; o >>= 1) {
        const long long v2 = __shfl_xor_sync(kFullMask, v, o);
        const int r2 = __shfl_xor_sync(kFullMask, row, o);
        if (v2 > v || (v2 == v && r2 < row)) { v = v2; row = r2; }
      }
      if (lane == 0) piv_s = v > 0 ? row : -1;
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr < 0) return false;
    if (pr != p) {
      for (int j = p + t; j <= n; j += blockDim.x) {
        double *a = j < n ? M + n * j : b;
        const double x = a[p];
        a[p] = a[pr];
        a[pr] = x;
      }
      __syncthreads();
    }
    const double d = M[p + n * p];
    const double sc = inv_pow2_exponent(fabs(d));
    const int m = n - p - 1;
    for (int e = t; e < m * (m + 1); e += blockDim.x) {
      const int i = p + 1 + e % m, j = p + 1 + e / m;  // j == n: the right-hand side
      double *col = j < n ? M + n * j : b;
      col[i] = (d * col[i] - M[i + n * p] * col[p]) * sc;
    }
    __syncthreads();
  }
  for (int k = t; k < n; k += blockDim.x) rdiag[k] = 1.0 / M[k + n * k];
  __syncthreads();
  if (t < 32) {  // back substitution, lanes = rows
    double x = lane < n ? b[lane] : 0.0;
    for (int k = n - 1; k >= 0; --k) {
      const double xk = __shfl_sync(kFullMask, x, k) * rdiag[k];
      if (lane == k) x = xk;
      if (lane < k) x -= M[lane + n * k] * xk;
    }
    if (lane < n) b[lane] = x;
  }
  __syncthreads();
  return true;
}

// Block argmax with the tie rule: the lowest index whose value is within a
// relative kTieRel of the maximum.  val < 0 marks excluded entries.
__device__ int block_argmax_tie(const double *val, int n) {
  __shared__ double red_d[32];
  __shared__ int red_i[32];
  double m = -1.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, val[k]);
  m = block_max(m, red_d);
  const double thr = m * (1.0 - kTieRel);
  int best = 0x7fffffff;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (val[k] >= 0.0 && val[k] >= thr) best = min(best, k);
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFullMask, best, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red_i[threadIdx.x >> 5] = best;
  __syncthreads();
  int b = 0x7fffffff;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) b = min(b, red_i[w]);
  __syncthreads();
  return b;
}

// ------------------------------------------------------------------
// step 2: angle choice, one thread-block cluster per instance.  CTA g of the
// cluster owns angles [g*slice, (g+1)*slice) as columns of A = W0^T in its
// shared memory (row i of A at A + i*slice_max), each column worked on by a
// team of T threads (T a power of two, rows split by i mod T).  Per pivot
// step: (1) every CTA computes the remaining squared norm (or the squared
// DEIM interpolation residual) of its unused columns and its largest one;
// cluster barrier; (2) every CTA reads the CTAs' maxima and then all
// squared norms through distributed shared memory and takes the same pivot:
// the lowest angle whose norm is within a relative 1e-12 of the largest
// (reading R8); (3) in pivoted-QR mode every CTA reads the pivot column from
// its owner and applies the same Householder reflection to its unused
// columns.  Norms and maxima alternate between two buffers by step parity
// and chosen columns are never written again, so one cluster barrier per
// step suffices.  CTA 0 then forms What, beta, gamma = What^{-T} beta and
// C0 = S0 What^T.
// ------------------------------------------------------------------
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(256)
k_select(const Inst *__restrict__ insts, int slice_max) {
  pdl_wait();
  pdl_trigger();
  cg::cluster_group cluster = cg::this_cluster();
  const int g = (int)cluster.block_rank();
  const Inst &I = insts[blockIdx.x / kCl];
  const bool active = *I.status == kOk;  // read before the first barrier
  const int r = I.r, K = I.K;
  const int slice = (K + kCl - 1) / kCl, k0 = min(K, g * slice), k1 = min(K, k0 + slice);
  const int ns = k1 - k0;
  extern __shared__ double sh[];
  double *A = sh;                          // r x slice_max, A[i*slice_max + c]
  double *nrm = A + 32 * slice_max;        // [2][slice_max] squared norms
  unsigned char *used = reinterpret_cast<unsigned char *>(nrm + 2 * slice_max);
  __shared__ double v[32], col[32], M[32 * 32], rhs[32], bpart[32];
  __shared__ long long lmax[2], red_l[32];  // maxima as bit patterns
  __shared__ int sel[32];
  __shared__ int red_i[32];
  __shared__ double hh_s;
  __shared__ long long thr_s;
  const double *W = I.W0;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  // column teams: T threads per column, rows i = m, m + T, ...
  int T = 1;
  while (T < 32 && 2 * T * max(ns, 1) <= (int)blockDim.x) T *= 2;
  const int m = t & (T - 1), c_first = t / T, c_step = (int)blockDim.x / T;
  for (int e = t; e < r * ns; e += blockDim.x) {
    const int i = e / ns, c = e - i * ns;
    A[i * slice_max + c] = active ? W[(k0 + c) + (size_t)K * i] : 0.0;
  }
  for (int c = t; c < ns; c += blockDim.x) used[c] = 0;
  // this CTA's share of beta_j = sum_k w_k W0_kj
  for (int j = wid; j < r; j += nw) {
    double s = 0.0;
    if (active)
      for (int k = k0 + lane; k < k1; k += 32) s += I.w[k] * W[k + (size_t)K * j];
    s = warp_sum(s);
    if (lane == 0) bpart[j] = s;
  }
  __syncthreads();
  for (int s = 0; s < r; ++s) {
    const int par = s & 1;
    double *nr = nrm + par * slice_max;
    // (1) squared norms (or residuals) of the unused owned columns
    if (I.selection == 1 && s > 0) {
      // DEIM: interpolation coefficients on the s chosen points,
      // W0[sel, 0:s] c = W0[sel, s]
      for (int e = t; e < s * s; e += blockDim.x) {
        const int i = e % s, l = e / s;
        M[e] = active ? W[sel[i] + (size_t)K * l] : (i == l ? 1.0 : 0.0);
      }
      for (int i = t; i < s; i += blockDim.x) rhs[i] = active ? W[sel[i] + (size_t)K * s] : 0.0;
      __syncthreads();
      block_solve(M, rhs, s);  // a singular system leaves rhs partly reduced; the step goes on
    }
    for (int base = 0; base < ns; base += c_step) {  // the same trip count in every thread
      const int c = base + c_first < ns ? base + c_first : -1;
      double x = 0.0;
      if (c >= 0) {
        if (I.selection == 0) {
          for (int i = s + ((m - s) & (T - 1)); i < r; i += T) {
            const double a = A[i * slice_max + c];
            x += a * a;
          }
        } else {
          for (int i = m; i <= s; i += T) {
            const double a = A[i * slice_max + c];
            x += i == s ? a : -rhs[i] * a;
          }
        }
      }
      for (int o = T >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
      if (c >= 0 && m == 0) nr[c] = used[c] ? -1.0 : (I.selection == 0 ? x : x * x);
    }
    __syncthreads();
    // maxima on the bit patterns (squared norms are >= 0, unused columns
    // hold -1 and so a negative pattern): integer compares only
    long long mx = -1;
    for (int c = t; c < ns; c += blockDim.x) mx = max(mx, __double_as_longlong(nr[c]));
    mx = warp_max(mx);
    if (lane == 0) red_l[wid] = mx;
    __syncthreads();
    if (t == 0) {
      long long x = -1;
      for (int q = 0; q < nw; ++q) x = max(x, red_l[q]);
      lmax[par] = x;
    }
    cluster.sync();
    // (2) the same pivot in every CTA
    if (wid == 0) {
      long long x = lane < kCl ? cluster.map_shared_rank(lmax, lane)[par] : -1;
      x = warp_max(x);
      if (lane == 0) {
        const double g2 = x >= 0 ? __longlong_as_double(x) : -1.0;
        thr_s = __double_as_longlong(g2 * ((1.0 - kTieRel) * (1.0 - kTieRel)));  // on squared norms
      }
    }
    __syncthreads();
    const long long thr = thr_s;
    int best = 0x7fffffff;
    for (int k = t; k < K; k += blockDim.x) {
      const int o = k / slice;
      const double x = cluster.map_shared_rank(nrm, o)[par * slice_max + (k - o * slice)];
      if (thr >= 0 && __double_as_longlong(x) >= thr) best = min(best, k);
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFullMask, best, o));
    if (lane == 0) red_i[wid] = best;
    __syncthreads();
    if (t == 0) {
      int p = 0x7fffffff;
      for (int q = 0; q < nw; ++q) p = min(p, red_i[q]);
      if (p < 0 || p >= K) {  // no finite candidate (NaN input)
        if (active && g == 0) set_status(I.status, kESingular);
        p = 0;
      }
      sel[s] = p;
    }
    __syncthreads();
    const int p = sel[s], owner = p / slice, pl = p - owner * slice;
    if (owner == g && t == 0) used[pl] = 1;  // never written again
    if (I.selection == 0) {
      if (t < r) col[t] = cluster.map_shared_rank(A, owner)[t * slice_max + pl];
      __syncthreads();
      if (wid == 0) {  // Householder vector v of x = col[s..r), hh = 2 / v^T v
        const double ci = (lane >= s && lane < r) ? col[lane] : 0.0;
        const double ss = warp_sum(ci * ci);
        const double nrm_p = sqrt(ss);
        const double a = col[s] >= 0 ? -nrm_p : nrm_p;
        v[lane] = lane == s ? ci - a : ci;
        // v^T v = 2 (|x|^2 + |x_s| |x|)
        if (lane == 0) hh_s = ss > 0.0 ? 1.0 / fma(fabs(col[s]), nrm_p, ss) : 0.0;
      }
      __syncthreads();
      const double hh = hh_s;
      for (int base = 0; base < ns; base += c_step) {
        const int c0 = base + c_first;
        const int c = (c0 < ns && hh != 0.0 && !used[min(c0, ns - 1)]) ? c0 : -1;
        const int i0 = s + ((m - s) & (T - 1));
        double d = 0.0;
        if (c >= 0)
          for (int i = i0; i < r; i += T) d += v[i] * A[i * slice_max + c];
        for (int o = T >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(kFullMask, d, o);
        if (c >= 0) {
          const double f = d * hh;
          for (int i = i0; i < r; i += T) A[i * slice_max + c] -= f * v[i];
        }
      }
    }
    __syncthreads();
  }
  cluster.sync();  // every CTA's beta share is final
  if (g == 0 && active && t < r) {
    double x = 0.0;
    for (int q = 0; q < kCl; ++q) x += cluster.map_shared_rank(bpart, q)[t];
    rhs[t] = x;
  }
  cluster.sync();  // peers' shared memory stays valid until CTA 0 has read it
  if (!active || g != 0) return;
  // What_ij = W0_j(Om^(i)), beta, gamma = What^{-T} beta, C0 = S0 What^T
  double *What = I.small + I.lay.What;
  double *beta = I.small + I.lay.beta;
  for (int e = t; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    const double x = W[sel[i] + (size_t)K * j];
    What[e] = x;
    M[j + r * i] = x;  // What^T
  }
  for (int i = t; i < r; i += blockDim.x) {
    I.idx[i] = sel[i];
    beta[i] = rhs[i];
  }
  __syncthreads();
  if (!block_solve(M, rhs, r)) {
    if (t == 0) set_status(I.status, kESingular);
    return;
  }
  for (int i = t; i < r; i += blockDim.x) I.small[I.lay.gamma + i] = rhs[i];
  double *C0 = I.small + I.lay.C0;
  for (int e = t; e < r * r; e += blockDim.x) {
    const int k = e % r, j = e / r;
    double x = 0.0;
    for (int l = 0; l < r; ++l) x += I.S0[k + r * l] * What[j + r * l];
    C0[e] = x;
  }
}

// ------------------------------------------------------------------
// One CholeskyQR pass on G = scale * sum_c part[c] (r x r, c over the
// cluster partials): R upper triangular with R^T R = G (+ shift), by the
// division-free elimination of chol_core.cuh.  Modes:
//   1 first pass: unshifted Cholesky that also detects dependent columns
//     (residual^2 < tau_dep |column|^2).  Dependent columns are marked in
//     flag[2 + j] and counted in flag[1] (they are then replaced by
//     pseudo-random columns and the pass is redone in mode 4).  Without
//     dependent columns a failed pivot falls back to a shifted Cholesky
//     (shifted CholeskyQR) and sets flag[0] (a third pass is needed).
//   2 always: Cholesky, shifted if needed (sets flag[0] when shifted)
//   3 only if flag[0]; otherwise R = I
//   4 only if flag[1] (after the fill); as mode 2
// ------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_chol(const CholJob *__restrict__ jobs,
                                              const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const CholJob J = jobs[blockIdx.x];
  const Inst &I = insts[blockIdx.x];
  if (*I.status != kOk) return;
  __shared__ double G[32 * 32];
  __shared__ CholScratch S;
  const int r = J.r, t = threadIdx.x;
  int *flag = J.flag;
  const bool run = J.mode == 1 || J.mode == 2 || (J.mode == 3 && flag[0] != 0) ||
                   (J.mode == 4 && flag[1] != 0);
  if (!run) {
    if (J.mode == 3)
      for (int e = t; e < r * r; e += blockDim.x) J.R[e] = (e % r == e / r) ? 1.0 : 0.0;
    return;
  }
  for (int e = t; e < r * r; e += blockDim.x)
    S.C[e] = J.scale * sum_partials(J.part, J.nblocks, (size_t)r * r, e);
  __syncthreads();
  // symmetrise (both triangles hold the same sums up to rounding order)
  for (int e = t; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    G[e] = (i == j) ? S.C[e] : 0.5 * (S.C[i + r * j] + S.C[j + r * i]);
  }
  if (J.mode == 1 && t == 0) {
    flag[0] = 0;
    flag[1] = 0;
  }
  if (J.mode == 1 && t < 32) flag[2 + t] = 0;
  __syncthreads();
  int ndep;
  bool shifted;
  chol_core(G, r, J.mode == 1, J.u, J.tau_dep, J.R, S, &ndep, &shifted);
  if (ndep > 0) {
    // mark the dependent columns; the pass is redone after the fill
    if (t == 0) flag[1] = ndep;
    if (t < r) flag[2 + t] = S.dep[t];
    return;
  }
  if (shifted && t == 0) flag[0] = 1;
}

// ------------------------------------------------------------------
// step 7 operators from the reduced sums (unscaled) in small[G .. vec]
// ------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_proj_post(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (*I.status != kOk) return;
  const int r = I.r;
  double *s = I.small;
  const SmallLayout &L = I.lay;
  const double h2 = I.h2;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    const double g = s[L.G + e];
    s[L.Axp + e] = h2 / I.hx * (g - s[L.Nx + e]);
    s[L.Axm + e] = h2 / I.hx * (g - s[L.Nx + j + r * i]);
    s[L.Ayp + e] = h2 / I.hy * (g - s[L.Ny + e]);
    s[L.Aym + e] = h2 / I.hy * (g - s[L.Ny + j + r * i]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    s[L.Mt + e] *= h2;
    s[L.Ms + e] *= h2;
    s[L.P + e] *= h2;
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    s[L.vec + i] *= h2;                 // qh
    s[L.vec + r + i] *= I.hy;           // left edge
    s[L.vec + 2 * r + i] *= I.hy;       // right edge
    s[L.vec + 3 * r + i] *= I.hx;       // bottom edge
    s[L.vec + 4 * r + i] *= I.hx;       // top edge
  }
  __syncthreads();
  // PS0 = P S0
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double t = 0.0;
    for (int l = 0; l < r; ++l) t += s[L.P + i + r * l] * I.S0[l + r * j];
    s[L.PS0 + e] = t;
  }
}

// ------------------------------------------------------------------
// step 7, per angle (one warp per angle; lane j owns column j)
// ------------------------------------------------------------------
struct AngleOps {
  const double *Ax, *Ay, *bx, *by;
  double aox, aoy, px, py;
};

__device__ __forceinline__ AngleOps angle_ops(const Inst &I, const double *sm, int k) {
  const SmallLayout &L = I.lay;
  const int r = I.r;
  AngleOps o;
  const double ox = I.ox[k], oy = I.oy[k];
  o.Ax = sm + (ox > 0 ? 0 : r * r);          // smem copy: Axp, Axm, Ayp, Aym, ...
  o.Ay = sm + (oy > 0 ? 2 * r * r : 3 * r * r);
  const double *vec = sm + 6 * r * r;        // qh, bL, bR, bB, bT
  o.bx = vec + (ox > 0 ? r : 2 * r);
  o.by = vec + (oy > 0 ? 3 * r : 4 * r);
  o.aox = fabs(ox);
  o.aoy = fabs(oy);
  o.px = ox > 0 ? I.psi_edge[0] : (ox < 0 ? I.psi_edge[1] : 0.0);
  o.py = oy > 0 ? I.psi_edge[2] : (oy < 0 ? I.psi_edge[3] : 0.0);
  // a reflective edge's inflow is not prescribed: it enters through the
  // fixed point of k_refl_lstep (reading R19)
  if (I.reflect[ox > 0 ? 0 : 1]) o.px = 0.0;
  if (I.reflect[oy > 0 ? 2 : 3]) o.py = 0.0;
  (void)L;
  return o;
}

// Q_k[i] = qh_i + (P S0 W0_k)_i / (c dt) + |ox| psi_x bx_i + |oy| psi_y by_i
__device__ __forceinline__ double angle_q(const Inst &I, const double *sm, const AngleOps &o,
                                          int k, int i) {
  const int r = I.r;
  const double *PS0 = sm + 5 * r * r;
  const double *qh = sm + 6 * r * r;
  double t = 0.0;
  for (int l = 0; l < r; ++l) t += PS0[i + r * l] * I.W0[k + (size_t)I.K * l];
  return qh[i] + I.inv_cdt * t + o.aox * o.px * o.bx[i] + o.aoy * o.py * o.by[i];
}

// stage Axp, Axm, Ayp, Aym, Mt, PS0 (r x r each) and vec (5r) in smem
__device__ void stage_ops(const Inst &I, double *sm) {
  const int r = I.r;
  const SmallLayout &L = I.lay;
  const int offs[6] = {L.Axp, L.Axm, L.Ayp, L.Aym, L.Mt, L.PS0};
  for (int a = 0; a < 6; ++a)
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sm[a * r * r + e] = I.small[offs[a] + e];
  for (int e = threadIdx.x; e < 5 * r; e += blockDim.x) sm[6 * r * r + e] = I.small[L.vec + e];
  __syncthreads();
}

constexpr int kLsWarps = 4;

// step 7, per angle.  One warp per angle runs Gauss-Jordan elimination with
// partial pivoting on [B_k | I] (B_k padded to RB x RB with an identity
// block).  The 2 RB columns live in the warp's shared memory (column c at
// cols + c (RB + 1)); lane l updates columns l and l + 32, so every FP64
// instruction keeps the lanes busy, and the pivot steps form a run-time loop
// over an unrolled row update (small code, no instruction-cache misses).
// The identity half ends as B_k^{-1}: it is kept in lu for the last part of
// the L-step, y_k = B_k^{-1} Q_k goes to L, and the CTA accumulates
// sum w_k B_k^{-1} and sum w_k y_k (the C-bar device of Section 3.3).  CTA
// sums are added over the cluster through distributed shared memory;
// cluster c writes its partial (r^2 + r doubles) to partials + c*(r^2 + r).
template <int RB>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kLsWarps * 32)
k_lstep_angle(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  constexpr int NC = 2 * RB, LDC = RB + 1;
  const Inst &I = insts[blockIdx.y];
  if (rank_class(I.r) != RB) return;  // another launch serves this rank class
  const int nblk = I.lstep_blocks;
  if ((int)blockIdx.x >= nblk) return;  // whole clusters (nblk is a multiple of kCl)
  cg::cluster_group cluster = cg::this_cluster();
  const bool active = *I.status == kOk;
  extern __shared__ double sh[];
  const int r = I.r, K = I.K, rq = r * r + r;
  double *sm = sh;                              // staged operators, 6 r^2 + 5 r
  double *acc = sm + 6 * r * r + 5 * r;         // kLsWarps x (r^2 + r)
  double *colsw = acc + kLsWarps * rq;          // kLsWarps x NC x LDC
  double *part_s = colsw + kLsWarps * NC * LDC; // r^2 + r
  stage_ops(I, sm);
  for (int e = threadIdx.x; e < kLsWarps * rq; e += blockDim.x) acc[e] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double *myacc = acc + wid * rq;
  double *cols = colsw + wid * NC * LDC;
  const double *Mt = sm + 4 * r * r;
  const int gw = blockIdx.x * kLsWarps + wid, nwarps = nblk * kLsWarps;
  // with polar pairs (angles of polar cosines +-mu share Om_x, Om_y, hence
  // B_k, bit for bit) one elimination serves both angles of a pair
  const int na = I.n_azim, np2 = I.polar_pairs ? (K / na) / 2 : 0;
  const int items = I.polar_pairs ? np2 * na : K;
  for (int it = gw; active && it < items; it += nwarps) {
    const int k = it, kp = I.polar_pairs ? (K / na - 1 - it / na) * na + it % na : -1;
    const AngleOps o = angle_ops(I, sm, k);
    for (int c = lane; c < NC; c += 32) {
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        double v;
        if (c < RB) {
          if (c < r && i < r) v = o.aox * o.Ax[i + r * c] + o.aoy * o.Ay[i + r * c] + Mt[i + r * c];
          else v = (i == c) ? 1.0 : 0.0;
        } else {
          v = (i == c - RB) ? 1.0 : 0.0;
        }
        cols[c * LDC + i] = v;
      }
    }
    __syncwarp();
    bool singular = false;
    for (int p = 0; p < RB; ++p) {
      // pivot row: the largest |B_ip|, i >= p (integer compares, lowest row on ties)
      long long best = (lane >= p && lane < RB) ? abs_bits(cols[p * LDC + lane]) : -1;
      int pr = lane;
      for (int off = 16; off > 0; off >>= 1) {
        const long long b2 = __shfl_xor_sync(kFullMask, best, off);
        const int r2 = __shfl_xor_sync(kFullMask, pr, off);
        if (b2 > best || (b2 == best && r2 < pr)) { best = b2; pr = r2; }
      }
      if (best <= 0) { singular = true; break; }
      if (pr != p)
        for (int c = lane; c < NC; c += 32) {
          const double x = cols[c * LDC + p];
          cols[c * LDC + p] = cols[c * LDC + pr];
          cols[c * LDC + pr] = x;
        }
      __syncwarp();
      const double inv = 1.0 / cols[p * LDC + p];
      // row p scaled, the other rows eliminated; column p itself is not
      // needed any more and is left as it is
      for (int c = lane; c < NC; c += 32) {
        if (c == p) continue;
        double *col = cols + c * LDC;
        const double x = col[p] * inv;
#pragma unroll
        for (int i = 0; i < RB; ++i)
          if (i != p) col[i] -= cols[p * LDC + i] * x;
        col[p] = x;
      }
      __syncwarp();
    }
    if (singular) {
      if (lane == 0) set_status(I.status, kESingular);
      break;
    }
    // B_k^{-1} column j is cols column RB + j
    const double *binv = cols + RB * LDC;
    for (int u = 0; u < (kp >= 0 ? 2 : 1); ++u) {
      const int kk = u == 0 ? k : kp;
      const double qk = lane < r ? angle_q(I, sm, o, kk, lane) : 0.0;
      double y0 = 0.0, y1 = 0.0;
#pragma unroll
      for (int jj = 0; jj < RB; ++jj) {
        if (jj < r) {
          const double qj = __shfl_sync(kFullMask, qk, jj);
          if (lane < r) {
            const double t = binv[jj * LDC + lane] * qj;
            if (jj & 1) y1 += t; else y0 += t;
          }
        }
      }
      if (lane < r) {
        const double y = y0 + y1;
        I.L[(size_t)r * kk + lane] = y;
        myacc[r * r + lane] += I.w[kk] * y;
      }
      double *B = I.lu + (size_t)kk * r * r;
      for (int e = lane; e < r * r; e += 32) B[e] = binv[(e / r) * LDC + (e % r)];
    }
    const double wk = kp >= 0 ? I.w[k] + I.w[kp] : I.w[k];
    if (lane < r)
      for (int jj = 0; jj < r; ++jj) myacc[lane + r * jj] += wk * binv[jj * LDC + lane];
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rq; e += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kLsWarps; ++w) s += acc[w * rq + e];
    part_s[e] = s;
  }
  cluster.sync();
  const int rank = (int)cluster.block_rank(), share = (rq + kCl - 1) / kCl;
  double *out = I.partials + (size_t)(blockIdx.x / kCl) * rq;
  for (int e = rank * share + threadIdx.x; e < min(rq, (rank + 1) * share); e += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kCl; ++q) s += cluster.map_shared_rank(part_s, q)[e];
    out[e] = s;
  }
  cluster.sync();
}

// (I - Cbar M_s / 4pi) Lbar = zeta, tvec = M_s Lbar / 4pi
__global__ void __launch_bounds__(256) k_lstep_mid(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (*I.status != kOk) return;
  const int nparts = I.lstep_blocks / kCl;
  __shared__ double M[32 * 32], Cb[32 * 32], z[32], Lb[32];
  const int r = I.r;
  const SmallLayout &L = I.lay;
  for (int e = threadIdx.x; e < r * r + r; e += blockDim.x) {
    const double s = sum_partials(I.partials, nparts, (size_t)(r * r + r), e);
    if (e < r * r) Cb[e] = s; else z[e - r * r] = s;
  }
  __syncthreads();
  const double *Ms = I.small + L.Ms;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double t0 = 0.0, t1 = 0.0;
    for (int l = 0; l < r; l += 2) {
      t0 += Cb[i + r * l] * Ms[l + r * j];
      if (l + 1 < r) t1 += Cb[i + r * (l + 1)] * Ms[(l + 1) + r * j];
    }
    M[e] = (i == j ? 1.0 : 0.0) - (t0 + t1) / (4.0 * kPi);
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) Lb[i] = z[i];
  __syncthreads();
  if (!block_solve(M, Lb, r)) {
    if (threadIdx.x == 0) set_status(I.status, kESingular);
    return;
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    double t = 0.0;
    for (int l = 0; l < r; ++l) t += Ms[i + r * l] * Lb[l];
    I.small[L.tvec + i] = t / (4.0 * kPi);
    I.small[L.Lbar + i] = Lb[i];
  }
}

// L_k = B_k^{-1} (Q_k + M_s Lbar / 4pi) = y_k + B_k^{-1} tvec, one thread per
// entry (k, i) of L (angle-major rows of r)
__global__ void __launch_bounds__(256) k_lstep_back(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (I.refl_kap) return;  // reflective edges: k_refl_lstep forms L
  const int r = I.r, K = I.K;
  __shared__ double tv[32];
  if (threadIdx.x < r) tv[threadIdx.x] = I.small[I.lay.tvec + threadIdx.x];
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (*I.status != kOk || e >= K * r) return;
  const int k = e / r, i = e - k * r;
  const double *B = I.lu + (size_t)k * r * r;
  double s0 = 0.0, s1 = 0.0;
  for (int j = 0; j < r; j += 2) {
    s0 += B[i + r * j] * tv[j];
    if (j + 1 < r) s1 += B[i + r * (j + 1)] * tv[j + 1];
  }
  I.L[e] += s0 + s1;
}

// ------------------------------------------------------------------
// step 8: with Q (in W0) the orthonormal factor of M = diag(sqrt w) L^T,
// S = M^T Q (summed from the cross-Gram partials), so that L = S W^T with
// W = diag(1/sqrt w) Q; one-sided Jacobi SVD S = U Sigma V^T (descending),
// S0 <- Sigma, V and U kept for W <- W V and X <- X U, vphi = L w.
// ------------------------------------------------------------------
// mode 0: S0 <- S (no SVD; U = V = I), vphi; mode 1: SVD as well;
// mode 2: SVD of the stored S0 (canonical factors on request).
__global__ void __launch_bounds__(512) k_svd(const Inst *__restrict__ insts, int mode) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (*I.status != kOk) return;
  __shared__ double Uw[32 * 32], Vw[32 * 32], sv[32];
  __shared__ int ord[32];
  __shared__ int rot_s;
  const int r = I.r;
  const SmallLayout &L = I.lay;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    double t = 0.0;
    if (mode == 2) t = I.S0[e];
    else t = sum_partials(I.partials, I.angle_blocks / kCl, (size_t)r * r, e);  // one partial per cluster
    Uw[e] = t;  // S_ij = sum_k sqrt(w_k) L_ik Q_kj
    Vw[e] = (e % r == e / r) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (mode != 2) {  // vphi_i = sum_k w_k L_ik  (phi = X L w)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < r; i += nw) {
      double s = 0.0;
      for (int k = lane; k < I.K; k += 32) s += I.w[k] * I.L[(size_t)r * k + i];
      s = warp_sum(s);
      if (lane == 0) I.small[L.vphi + i] = s;
    }
  }
  if (mode == 0) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      I.S0[e] = Uw[e];
      const double d = (e % r == e / r) ? 1.0 : 0.0;
      I.small[L.U + e] = d;
      I.small[L.V + e] = d;
    }
    return;
  }
  // one-sided Jacobi; each sweep visits all pairs in n-1 rounds of n/2
  // disjoint pairs (circle method), one warp per pair.  A pair counts as
  // converged when |ga| <= 1e-14 sqrt(al be) or |ga| <= 1e-16 ||S||_F^2 (the
  // second keeps columns at rounding-noise level from rotating forever).
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = (r + 1) & ~1;
  __shared__ double red[32];
  double f2 = 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) f2 += Uw[e] * Uw[e];
  const double floor_ga = 1e-16 * block_sum(f2, red);
  (void)lane;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (threadIdx.x == 0) rot_s = 0;
    __syncthreads();
    for (int round = 0; round < n - 1; ++round) {
      for (int pr = wid; pr < n / 2; pr += nw) {
        // positions pr and n-1-pr of [0, rotate(1..n-1, round)]
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n - 1); };
        int i = player(pr), j = player(n - 1 - pr);
        if (i > j) { const int t = i; i = j; j = t; }
        if (j >= r) continue;
        const double ui = lane < r ? Uw[lane + r * i] : 0.0;
        const double uj = lane < r ? Uw[lane + r * j] : 0.0;
        const double al = warp_sum(ui * ui), be = warp_sum(uj * uj), ga = warp_sum(ui * uj);
        // converged pair: |ga| <= 1e-14 sqrt(al be), tested on squares
        if (fabs(ga) <= floor_ga || ga * ga <= 1e-28 * (al * be)) continue;
        if (lane == 0) rot_s = 1;
        // t = tan(theta), the smaller root of ga t^2 + (be - al) t - ga = 0,
        // written with one square root and one division (each several
        // hundred cycles in FP64 on this GPU), cos(theta) by a reciprocal
        // square root; t = 1 when be = al
        const double d = be - al;
        const double t = d == 0.0 ? 1.0
                                  : (d > 0.0 ? 2.0 * ga : -2.0 * ga) / (fabs(d) + sqrt(d * d + 4.0 * ga * ga));
        const double cs = rsqrt(1.0 + t * t), sn = cs * t;
        if (lane < r) {
          Uw[lane + r * i] = cs * ui - sn * uj;
          Uw[lane + r * j] = sn * ui + cs * uj;
          const double vi = Vw[lane + r * i], vj = Vw[lane + r * j];
          Vw[lane + r * i] = cs * vi - sn * vj;
          Vw[lane + r * j] = sn * vi + cs * vj;
        }
      }
      __syncthreads();
    }
    if (!rot_s) break;
  }
  if (threadIdx.x == 0) {
    for (int j = 0; j < r; ++j) {
      double t = 0.0;
      for (int k = 0; k < r; ++k) t += Uw[k + r * j] * Uw[k + r * j];
      sv[j] = sqrt(t);
      ord[j] = j;
    }
    for (int a = 1; a < r; ++a) {  // stable insertion sort, descending
      const int key = ord[a];
      int b = a - 1;
      while (b >= 0 && sv[ord[b]] < sv[key]) { ord[b + 1] = ord[b]; --b; }
      ord[b + 1] = key;
    }
  }
  __syncthreads();
  const double smax = sv[ord[0]];
  double *U = I.small + L.U, *V = I.small + L.V;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int k = e % r, j = e / r, o = ord[j];
    const double s = sv[o];
    V[k + r * j] = Vw[k + r * o];
    U[k + r * j] = (s > 1e-300 && s > 1e-15 * smax) ? Uw[k + r * o] / s : 0.0;
  }
  __syncthreads();
  // complete U columns of zero singular values (Gram-Schmidt on unit
  // vectors); the augmented step drops the columns from aug_r on
  if (threadIdx.x == 0) {
    const int keep = I.aug_r > 0 ? I.aug_r : r;
    for (int j = 0; j < keep; ++j) {
      double t = 0.0;
      for (int k = 0; k < r; ++k) t += U[k + r * j] * U[k + r * j];
      if (t > 0.5) continue;
      for (int e = 0; e < r; ++e) {
        double u[32];
        for (int k = 0; k < r; ++k) u[k] = k == e ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass)
          for (int l = 0; l < r; ++l) {
            if (l == j) continue;
            double d = 0.0, ll = 0.0;
            for (int k = 0; k < r; ++k) { d += U[k + r * l] * u[k]; ll += U[k + r * l] * U[k + r * l]; }
            if (ll < 0.5) continue;
            for (int k = 0; k < r; ++k) u[k] -= d * U[k + r * l];
          }
        double nn = 0.0;
        for (int k = 0; k < r; ++k) nn += u[k] * u[k];
        if (nn > 1e-2) {
          nn = sqrt(nn);
          for (int k = 0; k < r; ++k) U[k + r * j] = u[k] / nn;
          break;
        }
      }
    }
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    I.S0[e] = (i == j) ? sv[ord[j]] : 0.0;
  }
}

// ------------------------------------------------------------------
// augmented step (rank-2r basis truncated back to rank r)
// ------------------------------------------------------------------
// Before the rank-2r steps: S0 (2r x 2r) = [[S0_r, 0], [0, 0]] (X0 and W0 are
// stored with 2r columns whose last r stay zero).
__global__ void __launch_bounds__(256) k_aug_pad(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  const int m = I.r, r = I.aug_r;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    I.S0[e] = (i < r && j < r) ? I.S0_r[i + r * j] : 0.0;
  }
}

// After the SVD S = U Sigma V^T of the 2r x 2r S (k_svd mode 2): keep the r
// largest singular values.  With b = W^T w (W the step-8 angular basis),
// phi of the truncated factors is X^ (U_r Sigma_r V_r^T b): that vector goes
// to vphi for the temperature kernel; the columns r..2r-1 of U and V are
// zeroed, so the rotations X0 <- X^ U and W0 <- W V leave them zero; S0 and
// S0_r become diag(Sigma_r).
__global__ void __launch_bounds__(256) k_aug_trunc(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (*I.status != kOk) return;
  const int m = I.r, r = I.aug_r, K = I.K;
  __shared__ double b[32], y[32], sg[32];
  double *U = I.small + I.lay.U, *V = I.small + I.lay.V;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < m; j += nw) {
    double t = 0.0;
    for (int k = lane; k < K; k += 32) t += I.W0[(size_t)K * j + k] * I.w[k];
    t = warp_sum(t);
    if (lane == 0) b[j] = t;
  }
  if (threadIdx.x < m) sg[threadIdx.x] = I.S0[threadIdx.x * (m + 1)];
  __syncthreads();
  if (threadIdx.x < r) {
    double t = 0.0;
    for (int j = 0; j < m; ++j) t += V[j + m * threadIdx.x] * b[j];
    y[threadIdx.x] = sg[threadIdx.x] * t;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double t = 0.0;
    for (int i = 0; i < r; ++i) t += U[threadIdx.x + m * i] * y[i];
    I.small[I.lay.vphi + threadIdx.x] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    if (j >= r) {
      U[e] = 0.0;
      V[e] = 0.0;
    }
    I.S0[e] = (i == j && i < r) ? sg[i] : 0.0;
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    I.S0_r[e] = (i == j) ? sg[i] : 0.0;
  }
}

// Sign of W columns: the entry of largest magnitude (tie rule) made positive;
// the same flip is applied to U (and so to X in the temperature kernel).
__global__ void __launch_bounds__(256) k_sign(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (*I.status != kOk) return;
  extern __shared__ double val[];
  const int r = I.r, K = I.K;
  for (int j = 0; j < r; ++j) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) val[k] = fabs(I.W0[k + (size_t)K * j]);
    __syncthreads();
    const int am = block_argmax_tie(val, K);
    const bool flip = I.W0[am + (size_t)K * j] < 0.0;
    if (flip) {
      for (int k = threadIdx.x; k < K; k += blockDim.x) I.W0[k + (size_t)K * j] = -I.W0[k + (size_t)K * j];
      for (int i = threadIdx.x; i < r; i += blockDim.x) I.small[I.lay.U + i + r * j] *= -1.0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------
// host launchers (kernel attributes are set by prepare_small before any
// launch is captured into a graph)
// ------------------------------------------------------------------
static size_t select_smem(int slice_max) {
  return (size_t)(34 * slice_max) * sizeof(double) + (size_t)slice_max;
}
static int rank_bucket(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : 32; }
size_t lstep_angle_smem(int r) {
  const int RB = rank_bucket(r);
  return (size_t)(6 * r * r + 5 * r + kLsWarps * (r * r + r) + kLsWarps * 2 * RB * (RB + 1) + r * r + r) *
         sizeof(double);
}

cudaError_t prepare_small(int slice_max, int maxK, int rmax) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)select_smem(slice_max))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_lstep_angle<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)lstep_angle_smem(rmax))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_lstep_angle<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)lstep_angle_smem(rmax))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_lstep_angle<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)lstep_angle_smem(rmax))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_sign, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(maxK * sizeof(double)));
}
cudaError_t launch_select(const Inst *d, int n, int slice_max, cudaStream_t st) {
  return launch_pdl(k_select, dim3(n * kCl), dim3(256), select_smem(slice_max), st, d, slice_max);
}
cudaError_t launch_chol(const CholJob *dj, const Inst *d, int n, cudaStream_t st) {
  return launch_pdl(k_chol, dim3(n), dim3(256), 0, st, dj, d);
}
cudaError_t launch_proj_post(const Inst *d, int n, cudaStream_t st) {
  return launch_pdl(k_proj_post, dim3(n), dim3(256), 0, st, d);
}
// blocks: CTAs of the per-angle kernel (a multiple of kCl); maxK: most angles
// rmask: the rank classes present (one launch of the per-angle kernel each)
cudaError_t launch_lstep(const Inst *d, int n, int r_max, int rmask, int blocks, int maxK, cudaStream_t st) {
  const dim3 g(blocks, n);
  const size_t sm = lstep_angle_smem(r_max);
  cudaError_t e = cudaSuccess;
  if (rmask & 1) e = launch_pdl(k_lstep_angle<8>, g, dim3(kLsWarps * 32), sm, st, d);
  if (e == cudaSuccess && (rmask & 2)) e = launch_pdl(k_lstep_angle<16>, g, dim3(kLsWarps * 32), sm, st, d);
  if (e == cudaSuccess && (rmask & 4)) e = launch_pdl(k_lstep_angle<32>, g, dim3(kLsWarps * 32), sm, st, d);
  if (e != cudaSuccess) return e;
  if ((e = launch_pdl(k_lstep_mid, dim3(n), dim3(256), 0, st, d)) != cudaSuccess) return e;
  return launch_pdl(k_lstep_back, dim3((maxK * r_max + 255) / 256, n), dim3(256), 0, st, d);
}
cudaError_t launch_svd(const Inst *d, int n, int mode, cudaStream_t st) {
  return launch_pdl(k_svd, dim3(n), dim3(512), 0, st, d, mode);
}
cudaError_t launch_sign(const Inst *d, int n, int maxK, cudaStream_t st) {
  return launch_pdl(k_sign, dim3(n), dim3(256), (size_t)maxK * sizeof(double), st, d);
}

cudaError_t launch_aug_pad(const Inst *d, int n, cudaStream_t st) {
  return launch_pdl(k_aug_pad, dim3(n), dim3(256), 0, st, d);
}

cudaError_t launch_aug_trunc(const Inst *d, int n, cudaStream_t st) {
  return launch_pdl(k_aug_trunc, dim3(n), dim3(256), 0, st, d);
}

}  // namespace dlr
