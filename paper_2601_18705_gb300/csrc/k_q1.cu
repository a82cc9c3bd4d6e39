// k_q1.cu -- the SN-like DLR step (Algorithm 1) and the full-rank SN step on
// bilinear (Q1) elements: upwind DG with the Legendre basis 1, xi, eta,
// xi eta on each cell (Section 4.4's volume term G_j and face matrices F_d
// with the paper's bilinear elements).  "real" is the working precision of
// the O(N) work (float in mixed precision, double in FP64); the r x r and
// per-angle algebra of steps 2, 5, 7, 8 stays in FP64 as on DG0 cells.
//
// Storage.  A Q1 field has 4 coefficients per cell, row e = 4 c + m.  They
// are stored scaled by s = (1, 1/sqrt3, 1/sqrt3, 1/3): the scaled basis is
// orthonormal for (1/4) int int over the reference cell, so the L2 inner
// product of two Q1 fields is hx hy times the plain dot product of their 4 N
// stored rows.  Step 5 (CholeskyQR in the h^2 inner product) then runs
// unchanged over 4 N rows, and the cell's own coefficients are the stored
// ones divided by s.
//
//   k_q1_coeff      step 1 (per cell, as on DG0 cells) and step 3: psi0 at
//                   the chosen angles from X0 C0, the fixed sources
//                   q delta_m0 + psi0_j / (c dt), the starting phi, and the
//                   row weights sigma_t, sigma_s of the step-7 mass Grams
//   k_q1_sn_prep    the same for a full-rank SN instance (psi^n at every
//                   angle, phi^n = sum_k w_k psi^n_k)
//   k_q1_si         step 4: the collocation sweeps of the chosen angles and
//                   the source iteration, one cooperative launch; a sweep
//                   solves per cell the 4 x 4 upwind DG system, the upwind
//                   neighbours entering through their face traces (constant
//                   and slope)
//   k_q1_transport  the Q1 transport operator of one axis direction applied
//                   to every column of X (for the Galerkin operators of step
//                   7, summed by the cross Grams of k_tsgram)
//   k_q1_vec        step 7's q^ and unit-inflow edge vectors, then P S0
//   k_q1_tupdate    step 9: T from the cell average of phi = X (L w),
//                   X0 <- X U
//   k_q1_sn_tupdate the full-rank SN step's temperature update
#include <algorithm>

#include "dlr_internal.cuh"

namespace dlr {

namespace {

constexpr int kQ1Pub = 8;      // columns per progress publication
constexpr uint64_t kQ1WaitNs = 4000000000ull;
constexpr unsigned kQ1Full = 0xffffffffu;

// faces of the reference cell: xi = +1, xi = -1, eta = +1, eta = -1
enum Q1Face { kFR = 0, kFL = 1, kFT = 2, kFB = 3 };

}  // namespace

// Sweeping warps per CTA (bands in flight per angle): 16 in FP32; 8 in FP64,
// whose edge rows would not fit in shared memory at 16.
template <typename real>
struct Q1Cfg {
  static constexpr int NW = sizeof(real) == 4 ? 16 : 8;
};

// int over the reference cell of the squared basis function m
__device__ __forceinline__ double q1_mass(int m) { return m == 0 ? 4.0 : (m == 3 ? 4.0 / 9.0 : 4.0 / 3.0); }

// The trace of basis function i on a face, as (constant, slope along the
// face): on xi = +-1 the slope is in eta, on eta = +-1 in xi.
__device__ __forceinline__ void q1_basis_trace(int face, int i, double &t0, double &t1) {
  const double sg = (face == kFR || face == kFT) ? 1.0 : -1.0;
  if (face == kFR || face == kFL) {  // xi = sg: 1 -> 1, xi -> sg, eta -> eta, xi eta -> sg eta
    t0 = i == 0 ? 1.0 : (i == 1 ? sg : 0.0);
    t1 = i == 2 ? 1.0 : (i == 3 ? sg : 0.0);
  } else {                           // eta = sg: 1 -> 1, xi -> xi, eta -> sg, xi eta -> sg xi
    t0 = i == 0 ? 1.0 : (i == 2 ? sg : 0.0);
    t1 = i == 1 ? 1.0 : (i == 3 ? sg : 0.0);
  }
}
// The trace of the field u (unscaled coefficients) on a face.
template <typename real>
__device__ __forceinline__ void q1_trace(int face, const real *u, real &t0, real &t1) {
  t0 = real(0);
  t1 = real(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double a0, a1;
    q1_basis_trace(face, i, a0, a1);
    if (a0 != 0.0) t0 += real(a0) * u[i];
    if (a1 != 0.0) t1 += real(a1) * u[i];
  }
}
// int_{-1}^{1} (c0 + c1 s)(d0 + d1 s) ds
__device__ __forceinline__ double q1_face_int(double c0, double c1, double d0, double d1) {
  return 2.0 * c0 * d0 + (2.0 / 3.0) * c1 * d1;
}

// The transport part of the cell matrix of direction (ox, oy) on a cell of
// half-widths a, b (A[i + 4 j], test function i, trial function j): the
// volume term -int u (Om . grad v) and the outflow faces
// |Om . n| (face length / 2) int trace_i trace_j.  The reference-cell
// integrals of (d v_i / d xi) v_j are 4 for (i, j) = (1, 0) and 4/3 for
// (3, 2); of (d v_i / d eta) v_j, 4 for (2, 0) and 4/3 for (3, 1).
__device__ __forceinline__ void q1_cell_matrix(double ox, double oy, double a, double b, double *A) {
#pragma unroll
  for (int e = 0; e < 16; ++e) A[e] = 0.0;
  A[1 + 4 * 0] -= ox * b * 4.0;
  A[3 + 4 * 2] -= ox * b * (4.0 / 3.0);
  A[2 + 4 * 0] -= oy * a * 4.0;
  A[3 + 4 * 1] -= oy * a * (4.0 / 3.0);
  const int fx = ox >= 0 ? kFR : kFL, fy = oy >= 0 ? kFT : kFB;
  const double cx = fabs(ox) * b, cy = fabs(oy) * a;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double xi0, xi1, xj0, xj1, yi0, yi1, yj0, yj1;
      q1_basis_trace(fx, i, xi0, xi1);
      q1_basis_trace(fx, j, xj0, xj1);
      q1_basis_trace(fy, i, yi0, yi1);
      q1_basis_trace(fy, j, yj0, yj1);
      A[i + 4 * j] += cx * q1_face_int(xi0, xi1, xj0, xj1) + cy * q1_face_int(yi0, yi1, yj0, yj1);
    }
}
// The inflow coefficients: the terms |Om . n| (length / 2) int u_in trace_i
// of the traces (ux0, ux1), (uy0, uy1) entering through the upwind x- and
// y-faces are Fx[i] ux0 + Gx[i] ux1 + Fy[i] uy0 + Gy[i] uy1.
__device__ __forceinline__ void q1_inflow_coef(double ox, double oy, double a, double b, double *Fx, double *Gx,
                                               double *Fy, double *Gy) {
  const int fx = ox >= 0 ? kFL : kFR, fy = oy >= 0 ? kFB : kFT;
  const double cx = fabs(ox) * b, cy = fabs(oy) * a;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double x0, x1, y0, y1;
    q1_basis_trace(fx, i, x0, x1);
    q1_basis_trace(fy, i, y0, y1);
    Fx[i] = cx * 2.0 * x0;
    Gx[i] = cx * (2.0 / 3.0) * x1;
    Fy[i] = cy * 2.0 * y0;
    Gy[i] = cy * (2.0 / 3.0) * y1;
  }
}
// A x = r for the 4 x 4 cell matrix by division-free elimination: row i
// becomes d_p row_i - a_ip row_p (no pivoting: the symmetric part of an
// upwind DG cell matrix is positive definite -- half the inflow and outflow
// face terms plus the reaction -- so no pivot vanishes), then the four
// reciprocals of the diagonal at once and the back substitution.  x
// overwrites r; A is destroyed.
template <typename real>
__device__ __forceinline__ void q1_solve4(real *A, real *r) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const real d = A[p + 4 * p];
#pragma unroll
    for (int i = p + 1; i < 4; ++i) {
      const real f = A[i + 4 * p];
#pragma unroll
      for (int j = p + 1; j < 4; ++j) A[i + 4 * j] = d * A[i + 4 * j] - f * A[p + 4 * j];
      r[i] = d * r[i] - f * r[p];
    }
  }
  real inv[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) inv[p] = real(1) / A[p + 4 * p];
#pragma unroll
  for (int p = 3; p >= 0; --p) {
    real x = r[p];
#pragma unroll
    for (int j = p + 1; j < 4; ++j) x -= A[p + 4 * j] * r[j];
    r[p] = x * inv[p];
  }
}

// ------------------------------------------------------------------
// steps 1 and 3
// ------------------------------------------------------------------
// One thread per cell: the coefficients, the weights of the mass Grams, and
// per chosen angle j and coefficient m: psi0 = sum_l X0(e, l) C0(l, j),
// s0_j(e) = q delta_m0 + psi0 / (c dt), phi(e) = sum_j gamma_j psi0_j(e).
template <typename real>
__global__ void __launch_bounds__(128) k_q1_coeff(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (!I.q1) return;
  __shared__ real C0s[kMaxRank * kMaxRank], gam[kMaxRank];
  const int r = I.r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) C0s[e] = real(I.small[I.lay.C0 + e]);
  for (int e = threadIdx.x; e < r; e += blockDim.x) gam[e] = real(I.small[I.lay.gamma + e]);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= I.N || *I.status != kOk) return;
  const CellCoef cf = cell_coefficients(I, c);
  I.B0[c] = cf.B;
  I.D[c] = cf.D;
  const double st = cf.sig + I.inv_cdt;
  as<real>(I.sig_t)[c] = real(st);
  as<real>(I.ss4)[c] = real(cf.ss / (4.0 * kPi));
  as<real>(I.q)[c] = real(cf.q);
  const size_t M = (size_t)4 * I.N;
  const real *X0 = as_c<real>(I.X0);
  real *s0 = as<real>(I.s0), *phi = as<real>(I.phi0);
  const real qr = real(cf.q), icdt = real(I.inv_cdt);
  for (int m = 0; m < 4; ++m) {
    const size_t e = (size_t)4 * c + m;
    I.q1_wt[e] = st;
    I.q1_ws[e] = cf.ss;
    real x[kMaxRank];
#pragma unroll
    for (int l = 0; l < kMaxRank; ++l) x[l] = l < r ? X0[e + M * l] : real(0);
    real ph = real(0);
    for (int j = 0; j < r; ++j) {
      real p0 = real(0);
#pragma unroll
      for (int l = 0; l < kMaxRank; ++l)
        if (l < r) p0 = fmadd(x[l], C0s[l + r * j], p0);
      s0[e + M * j] = fmadd(icdt, p0, m == 0 ? qr : real(0));
      ph = fmadd(gam[j], p0, ph);
    }
    phi[e] = ph;
  }
}

// Full-rank SN on Q1: psi (4 N x K, scaled) holds psi^n; the same
// coefficients, s0_k = q delta_m0 + psi^n_k / (c dt), phi^n = sum_k w_k psi^n_k.
template <typename real>
__global__ void __launch_bounds__(128) k_q1_sn_prep(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (!I.q1 || c >= I.N || *I.status != kOk) return;
  const CellCoef cf = cell_coefficients(I, c);
  I.B0[c] = cf.B;
  I.D[c] = cf.D;
  as<real>(I.sig_t)[c] = real(cf.sig + I.inv_cdt);
  as<real>(I.ss4)[c] = real(cf.ss / (4.0 * kPi));
  as<real>(I.q)[c] = real(cf.q);
  const size_t M = (size_t)4 * I.N;
  const real *psi = as_c<real>(I.Psi);
  real *s0 = as<real>(I.s0), *phi = as<real>(I.phi0);
  const real qr = real(cf.q), icdt = real(I.inv_cdt);
  for (int m = 0; m < 4; ++m) {
    const size_t e = (size_t)4 * c + m;
    real ph = real(0);
    for (int k = 0; k < I.K; ++k) {
      const real p = psi[e + M * k];
      s0[e + M * k] = fmadd(icdt, p, m == 0 ? qr : real(0));
      ph = fmadd(real(I.w[k]), p, ph);
    }
    phi[e] = ph;
  }
}

// ------------------------------------------------------------------
// step 4: collocation sweeps and source iteration
// ------------------------------------------------------------------
// Shared memory of k_q1_si: (NW + 1) edge rows of 2 x nx_max traces, the
// band progress counters, the active flags and the scalar-flux weights.
template <typename real>
__host__ __device__ inline size_t q1_si_smem_bytes(int nx_max, int bands_max, int n_inst, int gam_max) {
  return (size_t)(Q1Cfg<real>::NW + 1) * 2 * nx_max * sizeof(real) + (size_t)(bands_max + 3) / 4 * 4 * sizeof(int) +
         (size_t)(n_inst + 3) / 4 * 4 * sizeof(int) + (size_t)3 * n_inst * sizeof(double) +
         (size_t)gam_max * sizeof(real) + 16;
}

// The inputs of one cell of a sweep: sigma_t, sigma_s / 4pi, and the 4
// coefficients of phi and of the fixed source (16-byte vector loads in FP32,
// two 16-byte loads each in FP64).
template <typename real>
struct Q1In {
  real st, sv, p[4], s[4];
};
__device__ __forceinline__ void q1_ld4(const float *a, float *v) {
  const float4 x = *reinterpret_cast<const float4 *>(a);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void q1_ld4(const double *a, double *v) {
  const double2 x = reinterpret_cast<const double2 *>(a)[0], y = reinterpret_cast<const double2 *>(a)[1];
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}
__device__ __forceinline__ void q1_st4(float *a, const float *v) {
  *reinterpret_cast<float4 *>(a) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void q1_st4(double *a, const double *v) {
  reinterpret_cast<double2 *>(a)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2 *>(a)[1] = make_double2(v[2], v[3]);
}

template <typename real>
struct Q1Smem {
  real *edge;     // (NW + 1) x 2 x nx_max
  int *prog;      // per band: columns published
  int nx_max;
};

// Spins until band b's progress reaches `need` columns (bounded in time;
// leaves on the abort flag).  Called by one lane.
__device__ __forceinline__ bool q1_wait_prog(volatile int *prog, int b, int need, volatile int *abort_flag) {
  if (prog[b] >= need) return true;
  const uint64_t t0 = global_ns();
  unsigned spins = 0;
  while (prog[b] < need) {
    if ((++spins & 15u) == 0) {
      __nanosleep(32);
      if (*abort_flag) return false;
      if (global_ns() - t0 > kQ1WaitNs) return false;
    }
  }
  __threadfence_block();
  return true;
}

// The sweep of chosen angle j of instance I by one CTA: warp w takes the
// bands w, w + NW, ... of 32 rows (lane i = row i of the band, mirrored
// so that the direction points to +u, +v); lane i handles column u at step
// t = u + i.  The left neighbour's face trace stays in the lane's
// registers, the lower one comes from lane i - 1 by a shuffle, and lane 0
// takes it from the edge row the band below published.  Each lane loads
// its cell inputs two steps ahead.  Returns false (in every thread of the
// CTA) if a wait gave up.
template <typename real>
__device__ bool q1_sweep(const Inst &I, int j, const Q1Smem<real> &S, const real *pold, volatile int *abort_flag) {
  constexpr int NW = Q1Cfg<real>::NW;
  const int nx = I.nx, ny = I.ny, nb = (ny + 31) / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) S.prog[b] = 0;
  __syncthreads();
  const int k = I.idx[j];
  const double ox = I.ox[k], oy = I.oy[k];
  const double a = 0.5 * I.hx, bh = 0.5 * I.hy;
  const bool flx = ox < 0, fly = oy < 0;
  const real inx = real(ox > 0 ? I.psi_edge[0] : (ox < 0 ? I.psi_edge[1] : 0.0));
  const real iny = real(oy > 0 ? I.psi_edge[2] : (oy < 0 ? I.psi_edge[3] : 0.0));
  real A0[16], dm[4], Fx[4], Gx[4], Fy[4], Gy[4];
  {
    double Ad[16], f0[4], f1[4], f2[4], f3[4];
    q1_cell_matrix(ox, oy, a, bh, Ad);
    q1_inflow_coef(ox, oy, a, bh, f0, f1, f2, f3);
#pragma unroll
    for (int e = 0; e < 16; ++e) A0[e] = real(Ad[e]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      dm[m] = real(a * bh * q1_mass(m));
      Fx[m] = real(f0[m]);
      Gx[m] = real(f1[m]);
      Fy[m] = real(f2[m]);
      Gy[m] = real(f3[m]);
    }
  }
  // outflow traces: x-face (u0 + gx u1, u2 + gx u3), y-face
  // (u0 + gy u2, u1 + gy u3) with g = +1 on the +x / +y face, -1 opposite
  const real gx = real(ox >= 0 ? 1 : -1), gy = real(oy >= 0 ? 1 : -1);
  real us[4], sc[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    us[m] = real(q1_unscale(m));
    sc[m] = real(q1_scale(m));
  }
  const size_t M = (size_t)4 * I.N;
  const real *sig_t = as_c<real>(I.sig_t), *ss4 = as_c<real>(I.ss4);
  const real *s0 = as_c<real>(I.s0) + M * j;
  real *psi = as<real>(I.Psi) + M * j;
  volatile int *prog = S.prog;
  bool ok = true;
  for (int b = wid; b < nb && ok; b += NW) {
    const int v = b * 32 + lane;
    const bool row_ok = v < ny;
    const int iy = fly ? ny - 1 - v : v;
    const real *ein = S.edge + (size_t)((b + NW) % (NW + 1)) * 2 * S.nx_max;
    real *eout = S.edge + (size_t)(b % (NW + 1)) * 2 * S.nx_max;
    real ux0 = inx, ux1 = real(0);  // trace entering through the left face
    real ty0 = real(0), ty1 = real(0);  // this lane's last top trace
    // the inputs of column u of this lane's row (zero outside the mesh)
    auto load = [&](int u, Q1In<real> &in) {
      if (row_ok && u >= 0 && u < nx) {
        const int c = iy * nx + (flx ? nx - 1 - u : u);
        in.st = sig_t[c];
        in.sv = ss4[c];
        q1_ld4(pold + (size_t)4 * c, in.p);
        q1_ld4(s0 + (size_t)4 * c, in.s);
      }
    };
    Q1In<real> n1 = {}, n2 = {};
    load(-lane, n1);
    load(1 - lane, n2);
    for (int t = 0; t < nx + 31; ++t) {
      const Q1In<real> cur = n1;
      n1 = n2;
      load(t + 2 - lane, n2);
      if (b > 0 && t < nx && (t % kQ1Pub) == 0) {
        int w_ok = 1;
        if (lane == 0) w_ok = q1_wait_prog(prog, b - 1, min(nx, t + kQ1Pub), abort_flag) ? 1 : 0;
        w_ok = __shfl_sync(kQ1Full, w_ok, 0);
        if (!w_ok) { ok = false; break; }
      }
      const int u = t - lane;
      real uy0 = __shfl_up_sync(kQ1Full, ty0, 1), uy1 = __shfl_up_sync(kQ1Full, ty1, 1);
      if (lane == 0) {
        if (b == 0) { uy0 = iny; uy1 = real(0); }
        else if (u < nx) { uy0 = ein[u]; uy1 = ein[S.nx_max + u]; }
      }
      if (row_ok && u >= 0 && u < nx) {
        const int ix = flx ? nx - 1 - u : u;
        const int c = iy * nx + ix;
        real A[16], x[4];
#pragma unroll
        for (int e = 0; e < 16; ++e) A[e] = A0[e];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const real src = fmadd(cur.sv, cur.p[m], cur.s[m]) * us[m];
          A[m + 4 * m] = fmadd(cur.st, dm[m], A[m + 4 * m]);
          real rr = dm[m] * src;
          rr = fmadd(Fx[m], ux0, rr);
          rr = fmadd(Gx[m], ux1, rr);
          rr = fmadd(Fy[m], uy0, rr);
          x[m] = fmadd(Gy[m], uy1, rr);
        }
        q1_solve4(A, x);
        real xs[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) xs[m] = x[m] * sc[m];
        q1_st4(psi + (size_t)4 * c, xs);
        ux0 = fmadd(gx, x[1], x[0]);
        ux1 = fmadd(gx, x[3], x[2]);
        ty0 = fmadd(gy, x[2], x[0]);
        ty1 = fmadd(gy, x[3], x[1]);
        if (lane == 31) {
          eout[u] = ty0;
          eout[S.nx_max + u] = ty1;
        }
      }
      // lane 31 finished column t - 31: publish every kQ1Pub columns
      const int done = t - 30;
      if (lane == 31 && done > 0 && (done % kQ1Pub == 0 || done == nx)) {
        __threadfence_block();
        prog[b] = done;
      }
      __syncwarp();
    }
  }
  if (!ok) *abort_flag = 1;
  return __syncthreads_and(ok) != 0;
}

// The whole source iteration of a batch of Q1 instances, one cooperative
// launch: phase A sweeps every (instance, chosen angle) unit (units claimed
// from a counter), phase B forms phi = sum_j gamma_j psi_j per coefficient
// and the convergence maxima on the unscaled coefficients, phase C takes the
// same decision in every CTA (as k_si).
template <typename real>
__global__ void __launch_bounds__(Q1Cfg<real>::NW * 32) k_q1_si(const Inst *__restrict__ insts, SiCtl ctl) {
  extern __shared__ __align__(16) unsigned char q1sm[];
  Q1Smem<real> S;
  S.nx_max = ctl.nx_max;
  S.edge = reinterpret_cast<real *>(q1sm);
  size_t off = (size_t)(Q1Cfg<real>::NW + 1) * 2 * ctl.nx_max * sizeof(real);
  S.prog = reinterpret_cast<int *>(q1sm + off);
  off += (size_t)(ctl.bands_max + 3) / 4 * 4 * sizeof(int);
  int *active = reinterpret_cast<int *>(q1sm + off);
  off += (size_t)(ctl.n_inst + 3) / 4 * 4 * sizeof(int);
  double *relax = reinterpret_cast<double *>(q1sm + off);  // relaxation state, 3 per instance
  off += (size_t)3 * ctl.n_inst * sizeof(double);
  off = (off + 15) & ~size_t(15);
  real *gam = reinterpret_cast<real *>(q1sm + off);
  __shared__ int unit_s, n_active_s;
  volatile int *abort_flag = ctl.abort_flag;
  for (int i = threadIdx.x; i < ctl.n_inst; i += blockDim.x) {
    active[i] = (*insts[i].status == kOk) ? 1 : 0;
    relax_reset(relax + 3 * i);
  }
  __syncthreads();
  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) {
      int n = 0;
      for (int i = 0; i < ctl.n_inst; ++i) n += active[i];
      n_active_s = n;
    }
    __syncthreads();
    if (n_active_s == 0) break;
    // ---- phase A ----
    for (;;) {
      if (threadIdx.x == 0) unit_s = (int)atomicAdd(ctl.work + (it & 1), 1u);
      __syncthreads();
      const int u = unit_s;
      __syncthreads();
      if (u >= ctl.n_units) break;
      const SiUnit U = ctl.units[u];
      if (!active[U.inst]) continue;
      const Inst &I = insts[U.inst];
      const real *pold = as_c<real>((it & 1) ? I.phi1 : I.phi0);
      if (!q1_sweep<real>(I, U.angle, S, pold, abort_flag)) break;
    }
    if (!grid_barrier(ctl.bar, abort_flag)) break;
    // ---- phase B ----
    if (blockIdx.x == 0) {
      for (int i = threadIdx.x; i < ctl.n_inst; i += blockDim.x) {
        insts[i].conv[((it + 1) & 1) * 2 + 0] = 0ull;
        insts[i].conv[((it + 1) & 1) * 2 + 1] = 0ull;
      }
      if (threadIdx.x == 0) ctl.work[(it + 1) & 1] = 0u;
    }
    for (int i = 0; i < ctl.n_inst; ++i) {
      if (!active[i]) continue;
      const Inst &I = insts[i];
      const int r = I.r;
      const size_t M = (size_t)4 * I.N;
      const real *psi = as_c<real>(I.Psi);
      const real *pold = as_c<real>((it & 1) ? I.phi1 : I.phi0);
      real *pnew = as<real>((it & 1) ? I.phi0 : I.phi1);
      __syncthreads();
      for (int q = threadIdx.x; q < r; q += blockDim.x)
        gam[q] = real(I.gamma_ext ? I.gamma_ext[q] : I.small[I.lay.gamma + q]);
      __syncthreads();
      real dmax = real(0), pmax = real(0);
      const real om = real(I.gamma_ext ? 1.0 : relax[3 * i]);  // relaxation (DLR; 1: the plain iteration)
      for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < M; e += (size_t)gridDim.x * blockDim.x) {
        real acc = real(0);
        for (int q = 0; q < r; ++q) acc = fmadd(gam[q], psi[e + M * q], acc);
        const real us = real(q1_unscale((int)(e & 3)));
        const real po = pold[e];
        dmax = max(dmax, abs(acc - po) * us);
        pmax = max(pmax, abs(acc) * us);
        if (!isfinite(acc)) dmax = real(INFINITY);  // diverged (max() drops NaN)
        pnew[e] = om == real(1) ? acc : fmadd(om, acc - po, po);
      }
      dmax = warp_max(dmax);
      pmax = warp_max(pmax);
      if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(I.conv + (it & 1) * 2 + 0, (double)dmax);
        atomic_max_nonneg(I.conv + (it & 1) * 2 + 1, (double)pmax);
      }
    }
    if (!grid_barrier(ctl.bar, abort_flag)) break;
    // ---- phase C ----
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < ctl.n_inst; ++i) {
        if (!active[i]) continue;
        const Inst &I = insts[i];
        volatile unsigned long long *cv = I.conv + (it & 1) * 2;
        const double d = __longlong_as_double((long long)cv[0]);
        const double m = __longlong_as_double((long long)cv[1]);
        const int done_iters = it + 1;
        bool done;
        if (ctl.force_iters > 0) {
          if (done_iters >= ctl.force_iters) active[i] = 0;
          continue;
        }
        // DLR only (SN: gamma = w > 0); true: diverging even when relaxed
        const bool diverged = !I.gamma_ext && relax_track(d, m, relax + 3 * i);
        if (diverged || !(d <= 1.0e308)) {  // or a non-finite scalar flux
          done = true;
          if (blockIdx.x == 0) set_status(I.status, kENotConv);
        } else if (I.fixed_iters > 0) {
          done = done_iters >= I.fixed_iters;
        } else {
          done = d <= I.si_tol * m;
          if (!done && done_iters >= I.max_iter) {
            done = true;
            if (blockIdx.x == 0) set_status(I.status, kENotConv);
          }
        }
        if (done) {
          active[i] = 0;
          if (blockIdx.x == 0) {
            *I.iters = done_iters;
            atomicAdd(I.iters_total, (unsigned long long)done_iters);
          }
        }
      }
    }
    __syncthreads();
  }
  if (*abort_flag && blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < ctl.n_inst; ++i)
      if (active[i]) set_status(insts[i].status, kETimeout);
  }
}

// ------------------------------------------------------------------
// step 7: Galerkin operators
// ------------------------------------------------------------------
// V = T X for the transport operator T of axis direction dir (0: +x,
// 1: -x, 2: +y, 3: -y) with zero boundary inflow: per cell the cell matrix
// times the cell's coefficients minus the inflow terms of the upwind
// neighbour's trace.  Stored divided by s, so that the cross Gram
// sum_e Xs_i(e) Vs_j(e) of the stored rows is X_i^T T X_j.
template <typename real>
__global__ void __launch_bounds__(128) k_q1_transport(const Inst *__restrict__ insts, int dir) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (!I.q1 || c >= I.N || *I.status != kOk) return;
  const double ox = dir == 0 ? 1.0 : (dir == 1 ? -1.0 : 0.0), oy = dir == 2 ? 1.0 : (dir == 3 ? -1.0 : 0.0);
  const double a = 0.5 * I.hx, b = 0.5 * I.hy;
  real A0[16], F[4], G[4];
  {
    double Ad[16], fx[4], gx[4], fy[4], gy[4];
    q1_cell_matrix(ox, oy, a, b, Ad);
    q1_inflow_coef(ox, oy, a, b, fx, gx, fy, gy);
#pragma unroll
    for (int e = 0; e < 16; ++e) A0[e] = real(Ad[e]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      F[m] = real(dir < 2 ? fx[m] : fy[m]);
      G[m] = real(dir < 2 ? gx[m] : gy[m]);
    }
  }
  const int nx = I.nx, ny = I.ny, ix = c % nx, iy = c / nx;
  int nb = -1, face = kFR;
  if (dir == 0 && ix > 0) { nb = c - 1; face = kFR; }
  if (dir == 1 && ix < nx - 1) { nb = c + 1; face = kFL; }
  if (dir == 2 && iy > 0) { nb = c - nx; face = kFT; }
  if (dir == 3 && iy < ny - 1) { nb = c + nx; face = kFB; }
  const size_t M = (size_t)4 * I.N;
  const real *X = as_c<real>(I.X);
  real *V = as<real>(I.q1_v);
  for (int j = 0; j < I.r; ++j) {
    const real *Xj = X + M * j;
    real u[4], out[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) u[m] = Xj[(size_t)4 * c + m] * real(q1_unscale(m));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      real t = real(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) t = fmadd(A0[i + 4 * m], u[m], t);
      out[i] = t;
    }
    if (nb >= 0) {
      real un[4], t0, t1;
#pragma unroll
      for (int m = 0; m < 4; ++m) un[m] = Xj[(size_t)4 * nb + m] * real(q1_unscale(m));
      q1_trace(face, un, t0, t1);
#pragma unroll
      for (int i = 0; i < 4; ++i) out[i] -= F[i] * t0 + G[i] * t1;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) V[(size_t)4 * c + m + M * j] = out[m] * real(q1_unscale(m));
  }
}

// Per CTA b (of I.partial_blocks) and column j: sum_c q_c X_j(c, 0) over the
// CTA's cells (FP64, fixed order), into partials[b r + j].
template <typename real>
__global__ void __launch_bounds__(256) k_q1_qsum(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (!I.q1 || (int)blockIdx.x >= I.partial_blocks || *I.status != kOk) return;
  __shared__ double ws[8][kMaxRank];
  const int r = I.r, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const size_t M = (size_t)4 * I.N;
  const real *X = as_c<real>(I.X), *q = as_c<real>(I.q);
  double acc[kMaxRank];
#pragma unroll
  for (int j = 0; j < kMaxRank; ++j) acc[j] = 0.0;
  const int per = (I.N + I.partial_blocks - 1) / I.partial_blocks;
  const int c0 = blockIdx.x * per, c1 = min(I.N, c0 + per);
  for (int c = c0 + t; c < c1; c += blockDim.x) {
    const double qc = (double)q[c];
#pragma unroll
    for (int j = 0; j < kMaxRank; ++j)
      if (j < r) acc[j] += qc * (double)X[(size_t)4 * c + M * j];
  }
#pragma unroll
  for (int j = 0; j < kMaxRank; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kQ1Full, v, o);
    if (lane == 0) ws[wid][j] = v;
  }
  __syncthreads();
  if (t < r) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += ws[w][t];
    I.partials[(size_t)blockIdx.x * r + t] = s;
  }
}

// One CTA per instance: q^_j = hx hy sum over the partials of k_q1_qsum; the
// inflow vectors of a unit isotropic inflow on each edge, (face length) x
// the trace's constant summed along the edge (left: X0 - X1, right: X0 + X1,
// bottom: X0 - X2, top: X0 + X2, unscaled); then P S0 (P reduced before).
// Sums in FP64, in a fixed order.
template <typename real>
__global__ void __launch_bounds__(256) k_q1_vec(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.x];
  if (!I.q1 || *I.status != kOk) return;
  __shared__ double red[256];
  const int r = I.r, nx = I.nx, ny = I.ny, t = threadIdx.x;
  const size_t M = (size_t)4 * I.N;
  const real *X = as_c<real>(I.X);
  double *vec = I.small + I.lay.vec;
  auto block_sum = [&](double v) {
    red[t] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (t < s) red[t] += red[t + s];
      __syncthreads();
    }
    const double x = red[0];
    __syncthreads();
    return x;
  };
  for (int j = t; j < r; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < I.partial_blocks; ++b) s += I.partials[(size_t)b * r + j];
    vec[j] = I.h2 * s;
  }
  for (int j = 0; j < r; ++j) {
    const real *Xj = X + M * j;
    double l = 0.0, rr = 0.0;
    for (int iy = t; iy < ny; iy += blockDim.x) {
      const size_t cl = (size_t)4 * (iy * nx), cr = (size_t)4 * (iy * nx + nx - 1);
      l += (double)Xj[cl] - kQ1Sqrt3 * (double)Xj[cl + 1];
      rr += (double)Xj[cr] + kQ1Sqrt3 * (double)Xj[cr + 1];
    }
    l = block_sum(l);
    rr = block_sum(rr);
    double bo = 0.0, to = 0.0;
    for (int ix = t; ix < nx; ix += blockDim.x) {
      const size_t cb = (size_t)4 * ix, ct = (size_t)4 * ((ny - 1) * nx + ix);
      bo += (double)Xj[cb] - kQ1Sqrt3 * (double)Xj[cb + 2];
      to += (double)Xj[ct] + kQ1Sqrt3 * (double)Xj[ct + 2];
    }
    bo = block_sum(bo);
    to = block_sum(to);
    if (t == 0) {
      vec[r + j] = I.hy * l;
      vec[2 * r + j] = I.hy * rr;
      vec[3 * r + j] = I.hx * bo;
      vec[4 * r + j] = I.hx * to;
    }
  }
  const double *P = I.small + I.lay.P;
  for (int e = t; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double x = 0.0;
    for (int l = 0; l < r; ++l) x += P[i + r * l] * I.S0[l + r * j];
    I.small[I.lay.PS0 + e] = x;
  }
}

// ------------------------------------------------------------------
// step 9
// ------------------------------------------------------------------
// One thread per coefficient row: X0 <- X U, and in the rows m = 0 the
// temperature update with the cell average phi = X(4c, :) (L w).
template <typename real>
__global__ void __launch_bounds__(128) k_q1_tupdate(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (!I.q1) return;
  __shared__ real U[kMaxRank * kMaxRank], vp[kMaxRank];
  const int r = I.r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) U[e] = real(I.small[I.lay.U + e]);
  for (int e = threadIdx.x; e < r; e += blockDim.x) vp[e] = real(I.small[I.lay.vphi + e]);
  __syncthreads();
  const size_t M = (size_t)4 * I.N;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= M || *I.status != kOk) return;
  const real *X = as_c<real>(I.X);
  real *X0 = as<real>(I.X0);
  real x[kMaxRank];
  real phi = real(0);
#pragma unroll
  for (int i = 0; i < kMaxRank; ++i) {
    x[i] = i < r ? X[e + M * i] : real(0);
    if (i < r) phi = fmadd(x[i], vp[i], phi);
  }
  for (int j = 0; j < r; ++j) {
    real v = real(0);
#pragma unroll
    for (int i = 0; i < kMaxRank; ++i)
      if (i < r) v = fmadd(x[i], U[i + r * j], v);
    X0[e + M * j] = v;
  }
  if ((e & 3) != 0) return;
  const int c = (int)(e >> 2);
  const double T0 = I.T[c];
  const double T = T0 + I.dt * sigma_at(I, c, T0) * ((double)phi - 4.0 * kPi * I.B0[c]) / I.D[c];
  I.T[c] = T;
  if (!(T > 0.0)) {
    atomicAdd(I.nonpos, 1);
    if (!I.allow_nonpos) set_status(I.status, kENonPos);
  }
}

// Full-rank SN on Q1: T from the cell average of the last source
// iteration's phi.
template <typename real>
__global__ void __launch_bounds__(256) k_q1_sn_tupdate(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (!I.q1 || c >= I.N || *I.status != kOk) return;
  const int last = *I.iters - 1;  // iteration it writes phi1 (it even) or phi0 (odd)
  const real *phi = as_c<real>((last & 1) ? I.phi0 : I.phi1);
  const double T0 = I.T[c];
  const double T = T0 + I.dt * sigma_at(I, c, T0) * ((double)phi[(size_t)4 * c] - 4.0 * kPi * I.B0[c]) / I.D[c];
  I.T[c] = T;
  if (!(T > 0.0)) {
    atomicAdd(I.nonpos, 1);
    if (!I.allow_nonpos) set_status(I.status, kENonPos);
  }
}

// Rows of a 4 N x cols Q1 matrix between stored (scaled) and plain
// Legendre coefficients: to_plain = 1 divides by s, 0 multiplies.
template <typename T>
__global__ void k_q1_rescale(T *A, size_t rows, int cols, int to_plain) {
  const size_t total = rows * (size_t)cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)((e % rows) & 3);
    A[e] = T(A[e] * (to_plain ? q1_unscale(m) : q1_scale(m)));
  }
}

// ------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------
template <typename real>
cudaError_t launch_q1_coeff(const Inst *d, int n, int maxN, bool sn, cudaStream_t st) {
  const dim3 g((maxN + 127) / 128, n);
  return sn ? launch_pdl(k_q1_sn_prep<real>, g, dim3(128), 0, st, d)
            : launch_pdl(k_q1_coeff<real>, g, dim3(128), 0, st, d);
}

template <typename real>
size_t q1_si_smem(int nx_max, int bands_max, int n_inst, int gam_max) {
  return q1_si_smem_bytes<real>(nx_max, bands_max, n_inst, gam_max);
}

// CTAs of the cooperative Q1 source iteration that fit at once (0: none).
template <typename real>
int q1_si_max_grid(int nx_max, int bands_max, int n_inst, int gam_max) {
  const size_t smem = q1_si_smem_bytes<real>(nx_max, bands_max, n_inst, gam_max);
  if (cudaFuncSetAttribute(k_q1_si<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_q1_si<real>, Q1Cfg<real>::NW * 32, smem) !=
      cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <typename real>
cudaError_t launch_q1_si(const Inst *d, const SiCtl &ctl, int grid, cudaStream_t st) {
  const size_t smem = q1_si_smem_bytes<real>(ctl.nx_max, ctl.bands_max, ctl.n_inst, ctl.gam_max);
  cudaError_t e = cudaFuncSetAttribute(k_q1_si<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Q1Cfg<real>::NW * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_q1_si<real>, d, ctl);
}

template <typename real>
cudaError_t launch_q1_transport(const Inst *d, int n, int maxN, int dir, cudaStream_t st) {
  return launch_pdl(k_q1_transport<real>, dim3((maxN + 127) / 128, n), dim3(128), 0, st, d, dir);
}
template <typename real>
cudaError_t launch_q1_vec(const Inst *d, int n, int maxblocks, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_q1_qsum<real>, dim3(maxblocks, n), dim3(256), 0, st, d);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_q1_vec<real>, dim3(n), dim3(256), 0, st, d);
}
template <typename real>
cudaError_t launch_q1_tupdate(const Inst *d, int n, int maxN, bool sn, cudaStream_t st) {
  if (sn) return launch_pdl(k_q1_sn_tupdate<real>, dim3((maxN + 255) / 256, n), dim3(256), 0, st, d);
  return launch_pdl(k_q1_tupdate<real>, dim3((4 * maxN + 127) / 128, n), dim3(128), 0, st, d);
}
cudaError_t launch_q1_rescale(void *A, bool is_float, size_t rows, int cols, int to_plain, cudaStream_t st) {
  const size_t total = rows * (size_t)cols;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  if (is_float) k_q1_rescale<float><<<blocks, 256, 0, st>>>(static_cast<float *>(A), rows, cols, to_plain);
  else k_q1_rescale<double><<<blocks, 256, 0, st>>>(static_cast<double *>(A), rows, cols, to_plain);
  return cudaGetLastError();
}

#define Q1_INSTANTIATE(real)                                                                   \
  template cudaError_t launch_q1_coeff<real>(const Inst *, int, int, bool, cudaStream_t);      \
  template size_t q1_si_smem<real>(int, int, int, int);                                        \
  template int q1_si_max_grid<real>(int, int, int, int);                                       \
  template cudaError_t launch_q1_si<real>(const Inst *, const SiCtl &, int, cudaStream_t);     \
  template cudaError_t launch_q1_transport<real>(const Inst *, int, int, int, cudaStream_t);   \
  template cudaError_t launch_q1_vec<real>(const Inst *, int, int, cudaStream_t);              \
  template cudaError_t launch_q1_tupdate<real>(const Inst *, int, int, bool, cudaStream_t);
Q1_INSTANTIATE(float)
Q1_INSTANTIATE(double)
#undef Q1_INSTANTIATE

}  // namespace dlr
