// k_reflect.cu -- reflective edges in the SN-like DLR step (Algorithm 1
// with the general boundary conditions of Section 2.1; reading R19: a
// direction entering a reflective edge takes the value of its mirror
// direction in the same boundary cell).
//
//   k_refl_mats     What^{-1} (Gauss-Jordan), G = W0(Om_R(idx)) What^{-1} for
//                   the x and y mirror, H = C0 G^T (the first sweeps' inflow
//                   from X0)
//   k_refl_si_init  the reflective boundary cells' own fixed source kept in
//                   refl_base, the first sweeps' reflected inflow added to s0
//                   (the later sweeps' inflow is injected by the
//                   source-iteration kernel from G Psi)
//   k_refl_kap      What^{-1} Psi(c) in the boundary cells after step 4
//   k_refl_lstep    step 7 with the reflected inflow solved by a fixed point
//                   on the boundary values: the per-angle inverses B_k^{-1}
//                   and B_k^{-1} Q_k of k_lstep_angle are reused, each pass
//                   adds the extra inflow g_k, solves the C-bar system again
//                   and takes the boundary values from the new L.
#include "dlr_internal.cuh"

namespace dlr {

constexpr unsigned kReflMask = 0xffffffffu;
constexpr int kReflThreads = 256;
constexpr int kReflMaxPass = 5000;   // fixed-point passes of step 7
constexpr double kReflTol = 1e-14;   // relative change that ends them

// Inverse of the n x n matrix A (column-major in shared memory, destroyed)
// into X (shared memory) by Gauss-Jordan elimination with partial pivoting
// (largest magnitude, lowest row on ties).  Called by the whole CTA; returns
// false (in every thread) if a pivot is exactly zero.
__device__ bool block_invert(double *A, double *X, int n) {
  __shared__ int piv_s;
  __shared__ double mult[kMaxRank];
  const int t = threadIdx.x, lane = t & 31;
  for (int e = t; e < n * n; e += blockDim.x) X[e] = (e % n == e / n) ? 1.0 : 0.0;
  __syncthreads();
  for (int p = 0; p < n; ++p) {
    if (t < 32) {
      double v = (lane >= p && lane < n) ? fabs(A[lane + n * p]) : -1.0;
      int row = lane;
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(kReflMask, v, o);
        const int r2 = __shfl_xor_sync(kReflMask, row, o);
        if (v2 > v || (v2 == v && r2 < row)) { v = v2; row = r2; }
      }
      if (lane == 0) piv_s = v > 0 ? row : -1;
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr < 0) return false;
    if (pr != p)
      for (int j = t; j < 2 * n; j += blockDim.x) {
        double *col = j < n ? A + n * j : X + n * (j - n);
        const double x = col[p];
        col[p] = col[pr];
        col[pr] = x;
      }
    __syncthreads();
    const double inv = 1.0 / A[p + n * p];
    for (int i = t; i < n; i += blockDim.x) mult[i] = A[i + n * p];
    __syncthreads();
    for (int j = t; j < 2 * n; j += blockDim.x) {
      double *col = j < n ? A + n * j : X + n * (j - n);
      col[p] *= inv;
    }
    __syncthreads();
    for (int e = t; e < 2 * n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      if (i == p) continue;
      double *col = j < n ? A + n * j : X + n * (j - n);
      col[i] -= mult[i] * col[p];
    }
    __syncthreads();
  }
  return true;
}

__device__ __forceinline__ bool refl_any_x(const Inst &I) { return I.reflect[0] || I.reflect[1]; }
__device__ __forceinline__ bool refl_any_y(const Inst &I) { return I.reflect[2] || I.reflect[3]; }

// What^{-1}, RGx, RGy, RHx, RHy of every DLR instance with reflective edges
// (one CTA per instance).
__global__ void __launch_bounds__(kReflThreads) k_refl_mats(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (!I.refl_kap || *I.status != kOk) return;
  __shared__ double A[kMaxRank * kMaxRank], Wi[kMaxRank * kMaxRank], G[kMaxRank * kMaxRank];
  const int r = I.r, K = I.K;
  const SmallLayout &L = I.lay;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) A[e] = I.small[L.What + e];
  __syncthreads();
  if (!block_invert(A, Wi, r)) {
    if (threadIdx.x == 0) set_status(I.status, kESingular);
    return;
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) I.small[L.Winv + e] = Wi[e];
  const double *C0 = I.small + L.C0;
  for (int axis = 0; axis < 2; ++axis) {
    if (!(axis == 0 ? refl_any_x(I) : refl_any_y(I))) continue;
    // G_jm = sum_l W0(Om_R(idx_j))_l (What^{-1})_lm
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int j = e % r, m = e / r;
      const int km = mirror_angle(I.idx[j], I.n_azim, axis);
      double t = 0.0;
      for (int l = 0; l < r; ++l) t += I.W0[km + (size_t)K * l] * Wi[l + r * m];
      G[e] = t;
      I.small[(axis == 0 ? L.RGx : L.RGy) + e] = t;
    }
    __syncthreads();
    // H_lj = sum_m C0_lm G_jm: psi0 at the chosen angles is X0 C0, so the
    // first sweeps' inflow G Psi0(c) is X0(c) H
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int l = e % r, j = e / r;
      double t = 0.0;
      for (int m = 0; m < r; ++m) t += C0[l + r * m] * G[j + r * m];
      I.small[(axis == 0 ? L.RHx : L.RHy) + e] = t;
    }
    __syncthreads();
  }
}

// The first sweeps' reflected inflow from X0 H (entry e of refl_base, as in
// refl_inject; refl_base keeps the cell's own fixed source).
template <typename real>
__global__ void __launch_bounds__(kReflThreads) k_refl_si_init(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (!I.refl_kap || *I.status != kOk) return;
  const int L = I.ny + I.nx, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I.r * L) return;
  const int r = I.r, j = e / L, o = e - j * L;
  const ReflGeom<real> G(I, I.idx[j]);
  real *base = as<real>(I.refl_base) + (size_t)j * L;
  real *s0 = as<real>(I.s0) + (size_t)I.N * j;
  const real *X0 = as_c<real>(I.X0);
  auto first = [&](int c, int axis) {
    const double *H = I.small + (axis == 0 ? I.lay.RHx : I.lay.RHy) + (size_t)r * j;
    real v = real(0);
    for (int l = 0; l < r; ++l) v = fmadd(real(H[l]), X0[(size_t)I.N * l + c], v);
    return v;
  };
  if (o < I.ny) {
    if (!G.rx) return;
    const int c = o * I.nx + G.bx;
    const real f = s0[c];
    base[o] = f;
    real v = fmadd(G.ax, first(c, 0), f);
    if (G.ry && o == G.by) v = fmadd(G.ay, first(c, 1), v);
    s0[c] = v;
  } else {
    const int ix = o - I.ny;
    if (!G.ry || (G.rx && ix == G.bx)) return;
    const int c = G.by * I.nx + ix;
    const real f = s0[c];
    base[o] = f;
    s0[c] = fmadd(G.ay, first(c, 1), f);
  }
}

// Boundary slot s of the refl_kap rows: left edge rows 0 .. ny-1, right edge
// rows, bottom edge columns, top edge columns.
__device__ __forceinline__ int refl_slot_cell(const Inst &I, int s, int *edge) {
  const int nx = I.nx, ny = I.ny;
  if (s < ny) { *edge = 0; return s * nx; }
  s -= ny;
  if (s < ny) { *edge = 1; return s * nx + nx - 1; }
  s -= ny;
  if (s < nx) { *edge = 2; return s; }
  s -= nx;
  *edge = 3;
  return (ny - 1) * nx + s;
}
__device__ __forceinline__ int refl_slot_of(const Inst &I, int edge, int pos) {
  return edge == 0 ? pos : edge == 1 ? I.ny + pos : edge == 2 ? 2 * I.ny + pos : 2 * I.ny + I.nx + pos;
}

// refl_kap(s) = What^{-1} Psi(c_s) for the cells of reflective edges, one
// thread per (slot, component).
template <typename real>
__global__ void __launch_bounds__(kReflThreads) k_refl_kap(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (!I.refl_kap || *I.status != kOk) return;
  const int r = I.r, ns = 2 * (I.nx + I.ny), e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns * r) return;
  const int s = e / r, m = e - s * r;
  int edge = 0;
  const int c = refl_slot_cell(I, s, &edge);
  if (!I.reflect[edge]) return;
  const double *Wi = I.small + I.lay.Winv;
  const real *Psi = as_c<real>(I.Psi);
  double t = 0.0;
  for (int l = 0; l < r; ++l) t += Wi[m + r * l] * (double)Psi[(size_t)I.N * l + c];
  I.refl_kap[e] = t;
}

// The boundary cell of entry o of quadrature angle k (o < ny: row o of the
// x-edge the angle enters, else column o - ny of its y-edge), the edge, and
// whether it is reflective.
__device__ __forceinline__ bool refl_entry_of(const Inst &I, int k, int o, int *c, int *edge) {
  if (o < I.ny) {
    *edge = I.ox[k] > 0 ? 0 : 1;
    *c = o * I.nx + (*edge == 0 ? 0 : I.nx - 1);
  } else {
    *edge = I.oy[k] > 0 ? 2 : 3;
    *c = (*edge == 2 ? 0 : I.ny - 1) * I.nx + (o - I.ny);
  }
  return I.reflect[*edge] != 0;
}

// Step 7 with reflective edges, one cluster of kCl CTAs per instance.  On
// entry L holds y_k = B_k^{-1} Q_k, lu the inverses B_k^{-1} and partials
// the per-cluster sums of w_k B_k^{-1} and w_k y_k (k_lstep_angle).  The
// boundary values start from the collocation solution interpolated to the
// mirror angles, W0(Om_R) refl_kap; each pass then forms
//   g_k = sum_o f_o X(c_o) data(k, o)  (f = |Om_x| hy or |Om_y| hx),
//   u_k = B_k^{-1} g_k, zeta = zeta_0 + sum_k w_k u_k,
//   Lbar = (I - Cbar M_s / 4pi)^{-1} zeta, t = M_s Lbar / 4pi,
//   L_k = y_k + u_k + B_k^{-1} t,
//   data(k, o) = X(c_o) L_{R(k)},
// until the boundary values change by at most kReflTol of their largest
// magnitude.  All CTAs of the cluster take the same decisions (sums in a
// fixed order, each CTA solving the same r x r system).
template <typename real>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kReflThreads)
k_refl_lstep(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (!I.refl_kap) return;
  cg::cluster_group cluster = cg::this_cluster();
  if (*I.status != kOk) return;  // the same in every CTA of the cluster
  __shared__ double A[kMaxRank * kMaxRank], Minv[kMaxRank * kMaxRank], Ms[kMaxRank * kMaxRank];
  __shared__ double zeta0[kMaxRank], zp[kMaxRank], lb[kMaxRank], tv[kMaxRank];
  __shared__ double wsum[kReflThreads / 32][kMaxRank], part[kMaxRank];
  __shared__ double red[2][kReflThreads / 32], cmax[2];
  const int r = I.r, K = I.K, N = I.N, nx = I.nx, ny = I.ny, LB = nx + ny;
  const int rank = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kReflThreads / 32;
  const int gtid = rank * kReflThreads + threadIdx.x, gstride = kCl * kReflThreads;
  const int gw = rank * nw + wid, nwarps = kCl * nw;
  const SmallLayout &SL = I.lay;
  const real *X = as_c<real>(I.X);

  // Cbar, zeta_0 (partials in cluster order), M_s; (I - Cbar M_s / 4pi)^{-1}
  const int nparts = I.lstep_blocks / kCl, rq = r * r + r;
  for (int e = threadIdx.x; e < rq; e += blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += I.partials[(size_t)p * rq + e];
    if (e < r * r) Minv[e] = s;  // Cbar for now
    else zeta0[e - r * r] = s;
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Ms[e] = I.small[SL.Ms + e];
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double t = 0.0;
    for (int l = 0; l < r; ++l) t += Minv[i + r * l] * Ms[l + r * j];
    A[e] = (i == j ? 1.0 : 0.0) - t / (4.0 * kPi);
  }
  __syncthreads();
  const bool ok = block_invert(A, Minv, r);
  // boundary values from the collocation solution; y_k kept
  for (int e = gtid; e < K * LB; e += gstride) {
    const int k = e / LB, o = e - k * LB;
    int c, edge;
    if (!refl_entry_of(I, k, o, &c, &edge)) continue;
    const int km = mirror_angle(k, I.n_azim, o < ny ? 0 : 1);
    const double *kap = I.refl_kap + (size_t)r * refl_slot_of(I, edge, o < ny ? o : o - ny);
    double t = 0.0;
    for (int m = 0; m < r; ++m) t += I.W0[km + (size_t)K * m] * kap[m];
    I.refl_data[e] = t;
  }
  for (int e = gtid; e < K * r; e += gstride) I.refl_y[e] = I.L[e];
  cluster.sync();
  if (!ok) {
    if (rank == 0 && threadIdx.x == 0) set_status(I.status, kESingular);
    return;
  }

  int pass = 0;
  bool conv = false;
  for (; pass < kReflMaxPass && !conv; ++pass) {
    // (a) g_k and u_k = B_k^{-1} g_k, one warp per angle (lane i: component i)
    double acc = 0.0;
    for (int k = gw; k < K; k += nwarps) {
      const double fx = fabs(I.ox[k]) * I.hy, fy = fabs(I.oy[k]) * I.hx;
      const int ex = I.ox[k] > 0 ? 0 : 1, ey = I.oy[k] > 0 ? 2 : 3;
      const double *dk = I.refl_data + (size_t)k * LB;
      double g = 0.0;
      if (lane < r) {
        const real *Xi = X + (size_t)N * lane;
        if (I.reflect[ex]) {
          const int bx = ex == 0 ? 0 : nx - 1;
          for (int o = 0; o < ny; ++o) g += fx * (double)Xi[o * nx + bx] * dk[o];
        }
        if (I.reflect[ey]) {
          const int by0 = (ey == 2 ? 0 : ny - 1) * nx;
          for (int o = 0; o < nx; ++o) g += fy * (double)Xi[by0 + o] * dk[ny + o];
        }
      }
      const double *Bi = I.lu + (size_t)k * r * r;
      double u = 0.0;
      for (int j = 0; j < r; ++j) {
        const double gj = __shfl_sync(kReflMask, g, j);
        if (lane < r) u += Bi[lane + r * j] * gj;
      }
      if (lane < r) {
        I.refl_u[(size_t)k * r + lane] = u;
        acc += I.w[k] * u;
      }
    }
    if (lane < r) wsum[wid][lane] = acc;
    __syncthreads();
    if (threadIdx.x < r) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += wsum[w][threadIdx.x];
      part[threadIdx.x] = s;
    }
    cluster.sync();
    // (b) zeta, Lbar, t (each CTA alike)
    if (threadIdx.x < r) {
      double s = zeta0[threadIdx.x];
      for (int q = 0; q < kCl; ++q) s += cluster.map_shared_rank(part, q)[threadIdx.x];
      zp[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < r) {
      double s = 0.0;
      for (int l = 0; l < r; ++l) s += Minv[threadIdx.x + r * l] * zp[l];
      lb[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < r) {
      double s = 0.0;
      for (int l = 0; l < r; ++l) s += Ms[threadIdx.x + r * l] * lb[l];
      tv[threadIdx.x] = s / (4.0 * kPi);
    }
    __syncthreads();
    // (c) L_k = y_k + u_k + B_k^{-1} t
    for (int e = gtid; e < K * r; e += gstride) {
      const int k = e / r, i = e - k * r;
      const double *Bi = I.lu + (size_t)k * r * r;
      double s = 0.0;
      for (int j = 0; j < r; ++j) s += Bi[i + r * j] * tv[j];
      I.L[e] = I.refl_y[e] + I.refl_u[e] + s;
    }
    cluster.sync();  // every L_k written (and the peers' part read)
    // (d) new boundary values and their change
    double dmax = 0.0, vmax = 0.0;
    for (int e = gtid; e < K * LB; e += gstride) {
      const int k = e / LB, o = e - k * LB;
      int c, edge;
      if (!refl_entry_of(I, k, o, &c, &edge)) continue;
      const int km = mirror_angle(k, I.n_azim, o < ny ? 0 : 1);
      const double *Lm = I.L + (size_t)r * km;
      double t = 0.0;
      for (int i = 0; i < r; ++i) t += (double)X[(size_t)N * i + c] * Lm[i];
      dmax = fmax(dmax, fabs(t - I.refl_data[e]));
      vmax = fmax(vmax, fabs(t));
      I.refl_data[e] = t;
    }
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(kReflMask, dmax, o));
      vmax = fmax(vmax, __shfl_xor_sync(kReflMask, vmax, o));
    }
    if (lane == 0) {
      red[0][wid] = dmax;
      red[1][wid] = vmax;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double m = 0.0;
      for (int w = 0; w < nw; ++w) m = fmax(m, red[threadIdx.x][w]);
      cmax[threadIdx.x] = m;
    }
    cluster.sync();  // the new boundary values and every CTA's maxima
    double D = 0.0, V = 0.0;
    for (int q = 0; q < kCl; ++q) {
      const double *cm = cluster.map_shared_rank(cmax, q);
      D = fmax(D, cm[0]);
      V = fmax(V, cm[1]);
    }
    conv = D <= kReflTol * V;
    cluster.sync();  // the peers' maxima read before they are rewritten
  }
  if (rank == 0 && threadIdx.x == 0) {
    *I.refl_passes = pass;
    if (!conv) set_status(I.status, kENotConv);
  }
}

template <typename real>
cudaError_t launch_refl_pre(const Inst *d, int n, int maxr, int maxL, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_refl_mats, dim3(n), dim3(kReflThreads), 0, st, d);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_refl_si_init<real>, dim3((maxr * maxL + kReflThreads - 1) / kReflThreads, n),
                    dim3(kReflThreads), 0, st, d);
}

template <typename real>
cudaError_t launch_refl_kap(const Inst *d, int n, int maxr, int maxL, cudaStream_t st) {
  return launch_pdl(k_refl_kap<real>, dim3((2 * maxL * maxr + kReflThreads - 1) / kReflThreads, n),
                    dim3(kReflThreads), 0, st, d);
}

template <typename real>
cudaError_t launch_refl_lstep(const Inst *d, int n, cudaStream_t st) {
  return launch_pdl(k_refl_lstep<real>, dim3(kCl, n), dim3(kReflThreads), 0, st, d);
}

template cudaError_t launch_refl_pre<float>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_refl_pre<double>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_refl_kap<float>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_refl_kap<double>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_refl_lstep<float>(const Inst *, int, cudaStream_t);
template cudaError_t launch_refl_lstep<double>(const Inst *, int, cudaStream_t);

}  // namespace dlr
