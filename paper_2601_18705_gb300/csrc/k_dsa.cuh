// k_dsa.cuh -- diffusion synthetic acceleration (DSA) of the source
// iteration (Section 4.5), run inside the cooperative source-iteration
// launch of k_sweep.cu.
//
// After the sweeps at phi^l give phi^{l+1/2} = gamma^T Psi, the scalar flux
// becomes phi^{l+1} = phi^{l+1/2} + delta with
//   A delta = M_s (phi^{l+1/2} - phi^l),
//   A = (1/3) sum_j Fbar_j^T M_t^{-1} Fbar_j + F0 + M_a,
// the consistent diffusion operator of Section 4.5 on DG0 cells: the volume
// terms G_j vanish on piecewise constants, Fbar_j averages the face jumps
// (a centred difference), F0 penalises the jumps with
// kappa = (1/8 pi) sum_k w_k |Om_k . n| (the traditional penalty), and
// traces outside the domain are zero.  Scaled by 1/h^2 it is a 9-point cross
// stencil; for cell c and its neighbours c +- 1, c +- 2 along x (likewise
// along y, with nx for 1):
//   (A u)_c = d_c u_c - cx (ist_{c+1} u_{c+2} + ist_{c-1} u_{c-2})
//             - kx (u_{c+1} + u_{c-1}) - (y terms),
//   d_c     = sigma_a,c + 2 kx + 2 ky + cx (ist_{c+1} + ist_{c-1}) + (y terms),
// with cx = 1/(12 hx^2), kx = kappa_x / hx, ist = 1/sigma_t and
// sigma_a = sigma_t - sigma_s; a term whose cell c +- 1 (or c +- 2) is
// outside the mesh is dropped.  The right-hand side is sigma_s (phi^{l+1/2}
// - phi^l).
//
// The system is solved by Jacobi-preconditioned conjugate gradients, the
// search-direction update p = z + beta p_old evaluated inside the stencil
// pass (p in two buffers), so that one CG iteration is two passes and two
// grid barriers:
//   P1: p = z + beta p_old, q = A p, partial sums of p.q
//   P2: x += alpha p, r -= alpha q, z = r / d, partial sums of r.z, r.r
// CG scalars are sums of per-CTA partials that every CTA adds up itself in
// the same fixed order (one warp per instance), so all CTAs take the same
// decisions and the result does not depend on timing.
#pragma once

namespace dlr {

enum { kDsaPq = 0, kDsaRz = 1, kDsaRr = 2, kDsaBb = 3 };

constexpr double kFourPi = 12.566370614359172953850573533118;

// shared memory of the CG: 6 x n_inst scalars, then n_inst flags
__host__ __device__ inline size_t dsa_scalar_bytes(int n_inst, int dsa) {
  return dsa ? (size_t)6 * n_inst * sizeof(double) : 0;
}
__host__ __device__ inline size_t dsa_smem_bytes(int n_inst, int dsa) {
  return dsa ? dsa_scalar_bytes(n_inst, dsa) + (size_t)(n_inst + 3) / 4 * 4 * sizeof(int) : 0;
}

__device__ __forceinline__ double *dsa_slot(const SiCtl &ctl, int i, int slot) {
  return ctl.dsa_part + ((size_t)i * kDsaSlots + slot) * gridDim.x;
}

// Per-launch coefficients: 1/sigma_t, the diagonal d and 1/d.
template <typename real>
__device__ void dsa_setup(const Inst &I) {
  const real *st = as_c<real>(I.sig_t), *ss4 = as_c<real>(I.ss4);
  real *ist = as<real>(I.dsa_ist), *dg = as<real>(I.dsa_dg), *dinv = as<real>(I.dsa_dinv);
  real *p1 = as<real>(I.dsa_p1);
  const int nx = I.nx, ny = I.ny, N = I.N;
  const real cx = real(I.dsa_cx), cy = real(I.dsa_cy);
  const real k2 = real(2.0 * (I.dsa_kx + I.dsa_ky));
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int ix = c % nx, iy = c / nx;
    real d = st[c] - real(kFourPi) * ss4[c] + k2;
    if (ix + 1 < nx) d += cx / st[c + 1];
    if (ix > 0) d += cx / st[c - 1];
    if (iy + 1 < ny) d += cy / st[c + nx];
    if (iy > 0) d += cy / st[c - nx];
    ist[c] = real(1) / st[c];
    dg[c] = d;
    dinv[c] = real(1) / d;
    p1[c] = real(0);  // p_old of the first CG iteration (beta = 0 there)
  }
}

// Right-hand side of one DSA solve at cell c (called from the scalar-flux
// phase): r = b = sigma_s (phi_half - phi_old), x = 0, z = b / d; returns
// b.z and b.b through the accumulators.
template <typename real>
__device__ __forceinline__ void dsa_rhs(const Inst &I, int c, real phi_half, real phi_old,
                                        double &rz, double &bb) {
  const real b = real(kFourPi) * as_c<real>(I.ss4)[c] * (phi_half - phi_old);
  const real z = b * as_c<real>(I.dsa_dinv)[c];
  as<real>(I.dsa_x)[c] = real(0);
  as<real>(I.dsa_r)[c] = b;
  as<real>(I.dsa_z)[c] = z;
  rz += (double)b * (double)z;
  bb += (double)b * (double)b;
}

// out_s[i] = the sum over CTAs of partial slot s of instance i, for every
// instance with on[i] (slots s0 and s1 at once).
__device__ __forceinline__ void dsa_sum2(const SiCtl &ctl, const int *on, int s0, double *out0,
                                         int s1, double *out1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < ctl.n_inst; i += nw) {
    if (!on[i]) continue;
    const double *p0 = dsa_slot(ctl, i, s0), *p1 = dsa_slot(ctl, i, s1);
    // up to 8 partials per lane per round, all loads issued before the adds
    double v0 = 0, v1 = 0;
    for (int b0 = 0; b0 < (int)gridDim.x; b0 += 256) {
      double a0[8], a1[8];
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const int b = b0 + g * 32 + lane;
        const bool ok = b < (int)gridDim.x;
        a0[g] = ok ? p0[b] : 0.0;
        a1[g] = ok ? p1[b] : 0.0;
      }
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        v0 += a0[g];
        v1 += a1[g];
      }
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
      out0[i] = v0;
      out1[i] = v1;
    }
  }
  __syncthreads();
}

// P1 of one instance: u = z + beta p_old (u = z in the first iteration),
// then q = A u, p = u.  A warp takes 32 cells of one row (lane = x offset):
// the x-neighbours come from its lanes by shuffles plus a halo of four cells
// (x0 - 2, x0 - 1, x0 + 32, x0 + 33) loaded by lanes 0-3, the y-neighbours
// from the rows above and below; a cell outside the mesh counts as 0 (u and
// 1/sigma_t), which drops exactly the terms the stencil drops.
template <typename real>
struct DsaP1 {
  const real *__restrict__ z;
  const real *__restrict__ po;
  const real *__restrict__ ist;
  const real *__restrict__ dg;
  real *__restrict__ pn;
  real *__restrict__ q;
  int nx, ny;
  real beta, cx, cy, kx, ky;

  // The values one lane loads for one 32-cell segment (row iy, cells x0 ..
  // x0 + 31), gathered before any of them is used so that the loads of
  // several segments are in flight together.
  struct Seg {
    int c;       // this lane's cell (valid only if in)
    bool in;     // this lane's cell is inside the mesh
    real uc, ic, uh, ih, un1, un2, us1, us2, in1, is1, dc;
  };
  // u = z + beta p_old at cell c if ok, else 0 (p_old is zero before the
  // first iteration, where beta = 0)
  __device__ __forceinline__ real u(bool ok, int c) const {
    return ok ? fmadd(beta, po[c], z[c]) : real(0);
  }
  __device__ __forceinline__ void load(Seg &S, int iy, int x0) const {
    const int lane = threadIdx.x & 31, ix = x0 + lane;
    // row tests are the same for the whole warp
    const bool r0 = (unsigned)iy < (unsigned)ny;
    const bool rn1 = r0 && iy >= 1, rn2 = r0 && iy >= 2;
    const bool rs1 = r0 && iy + 1 < ny, rs2 = r0 && iy + 2 < ny;
    const bool col = ix < nx;
    const int c = iy * nx + ix;
    // halo cells of lanes 0-3: x0 - 2, x0 - 1, x0 + 32, x0 + 33
    const int hd = lane < 2 ? -2 : 30;  // offset of the halo cell from ix
    const int hx = ix + hd;
    const bool hok = r0 && lane < 4 && (unsigned)hx < (unsigned)nx;
    S.c = c;
    S.in = r0 && col;
    S.uc = u(S.in, c);
    S.ic = S.in ? ist[c] : real(0);
    S.uh = u(hok, c + hd);
    S.ih = hok ? ist[c + hd] : real(0);
    S.un1 = u(rn1 && col, c - nx);
    S.un2 = u(rn2 && col, c - 2 * nx);
    S.us1 = u(rs1 && col, c + nx);
    S.us2 = u(rs2 && col, c + 2 * nx);
    S.in1 = rn1 && col ? ist[c - nx] : real(0);
    S.is1 = rs1 && col ? ist[c + nx] : real(0);
    S.dc = S.in ? dg[c] : real(0);
  }
  // q = A u and p = u for the segment; returns this lane's u q (0 outside)
  __device__ __forceinline__ double finish(const Seg &S) const {
    const int lane = threadIdx.x & 31;
    real um1 = __shfl_up_sync(0xffffffffu, S.uc, 1), um2 = __shfl_up_sync(0xffffffffu, S.uc, 2);
    real up1 = __shfl_down_sync(0xffffffffu, S.uc, 1), up2 = __shfl_down_sync(0xffffffffu, S.uc, 2);
    real im1 = __shfl_up_sync(0xffffffffu, S.ic, 1), ip1 = __shfl_down_sync(0xffffffffu, S.ic, 1);
    const real h0 = __shfl_sync(0xffffffffu, S.uh, 0), h1 = __shfl_sync(0xffffffffu, S.uh, 1);
    const real h2 = __shfl_sync(0xffffffffu, S.uh, 2), h3 = __shfl_sync(0xffffffffu, S.uh, 3);
    const real g1 = __shfl_sync(0xffffffffu, S.ih, 1), g2 = __shfl_sync(0xffffffffu, S.ih, 2);
    if (lane == 0) {
      um1 = h1;
      um2 = h0;
      im1 = g1;
    }
    if (lane == 1) um2 = h1;
    if (lane == 30) up2 = h2;
    if (lane == 31) {
      up1 = h2;
      up2 = h3;
      ip1 = g2;
    }
    real off = kx * (up1 + um1);
    off = fmadd(cx, fmadd(ip1, up2, im1 * um2), off);
    off = fmadd(ky, S.us1 + S.un1, off);
    off = fmadd(cy, fmadd(S.is1, S.us2, S.in1 * S.un2), off);
    const real Au = fmadd(S.dc, S.uc, -off);
    if (S.in) {
      pn[S.c] = S.uc;
      q[S.c] = Au;
    }
    return (double)S.uc * (double)Au;
  }
};

// Block-wide sums of two values at once (one pair of barriers); every
// thread gets both.  scratch >= 64 entries.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) {
    scratch[wid] = a;
    scratch[32 + wid] = b;
  }
  __syncthreads();
  a = warp_sum(lane < nw ? scratch[lane] : 0.0);
  b = warp_sum(lane < nw ? scratch[32 + lane] : 0.0);
}

template <typename real> struct DsaVec;
template <> struct DsaVec<float> {
  using type = float4;
  static constexpr int kN = 4;
};
template <> struct DsaVec<double> {
  using type = double2;
  static constexpr int kN = 2;
};

// P2 on elements [0, n): x += a p, r -= a q, z = r dinv; accumulates r.z and r.r
template <typename real>
__device__ __forceinline__ void dsa_p2_elem(real a, real p, real qq, real &x, real &r, real &z,
                                            real dinv, double &rz, double &rr) {
  x = fmadd(a, p, x);
  r = fmadd(-a, qq, r);
  z = r * dinv;
  rz += (double)r * (double)z;
  rr += (double)r * (double)r;
}

// The CG solves of all instances with on[i] (set by the caller: active, DSA
// on, right-hand side nonzero), started from the partials of the scalar-flux
// phase.  sc: 6 x n_inst doubles of shared memory.  Returns false if a grid
// barrier gave up.
template <typename real>
__device__ __noinline__ bool dsa_solve(const Inst *__restrict__ insts, const SiCtl &ctl, int *on,
                                       double *sc, volatile int *abort_flag) {
  __shared__ double red[64];
  const int n = ctl.n_inst;
  double *rz = sc, *beta = sc + n, *alpha = sc + 2 * n, *bb = sc + 3 * n, *t0 = sc + 4 * n,
         *t1 = sc + 5 * n;
  dsa_sum2(ctl, on, kDsaRz, rz, kDsaBb, bb);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (!on[i]) continue;
    beta[i] = 0.0;
    if (!(bb[i] > 0.0)) on[i] = 0;  // phi did not change where sigma_s > 0: delta = 0
  }
  __syncthreads();
  for (int k = 0;; ++k) {
    bool any = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) any = any || on[i];
    if (!__syncthreads_or(any)) break;

    // P1: p = z + beta p_old, q = A p
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      const Inst &I = insts[i];
      DsaP1<real> P;
      P.z = as_c<real>(I.dsa_z);
      P.po = as_c<real>((k & 1) ? I.dsa_p0 : I.dsa_p1);
      P.ist = as_c<real>(I.dsa_ist);
      P.dg = as_c<real>(I.dsa_dg);
      P.pn = as<real>((k & 1) ? I.dsa_p1 : I.dsa_p0);
      P.q = as<real>(I.dsa_q);
      P.nx = I.nx;
      P.ny = I.ny;
      P.beta = k == 0 ? real(0) : real(beta[i]);
      P.cx = real(I.dsa_cx);
      P.cy = real(I.dsa_cy);
      P.kx = real(I.dsa_kx);
      P.ky = real(I.dsa_ky);
      const int nxb = (I.nx + 31) >> 5, items = I.ny * nxb;
      double pq = 0;
      // kSegs row segments per warp and round, all loads before any use (8 in
      // FP32; FP64 spills at 8)
      constexpr int kSegs = sizeof(real) == 4 ? 8 : 4;
      for (int t = gw; t < items; t += kSegs * warps) {
        typename DsaP1<real>::Seg S[kSegs];
#pragma unroll
        for (int g = 0; g < kSegs; ++g) {
          const int tg = t + g * warps;
          const int iy = tg / nxb;
          // a segment past the end loads nothing (its row is outside the mesh)
          P.load(S[g], tg < items ? iy : -8, (tg - iy * nxb) << 5);
        }
#pragma unroll
        for (int g = 0; g < kSegs; ++g) pq += P.finish(S[g]);
      }
      pq = block_sum(pq, red);
      if (threadIdx.x == 0) dsa_slot(ctl, i, kDsaPq)[blockIdx.x] = pq;
    }
    if (!grid_barrier(ctl.bar, abort_flag)) return false;

    // P2: x += alpha p, r -= alpha q, z = r / d
    dsa_sum2(ctl, on, kDsaPq, t0, kDsaPq, t1);
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (on[i]) alpha[i] = t0[i] != 0.0 ? rz[i] / t0[i] : 0.0;
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      const Inst &I = insts[i];
      const int N = I.N;
      const real *pn = as_c<real>((k & 1) ? I.dsa_p1 : I.dsa_p0);
      const real *q = as_c<real>(I.dsa_q), *dinv = as_c<real>(I.dsa_dinv);
      real *x = as<real>(I.dsa_x), *r = as<real>(I.dsa_r), *z = as<real>(I.dsa_z);
      const real a = real(alpha[i]);
      double prz = 0, prr = 0;
      // vectors of kN elements (the arrays are separate allocations, aligned),
      // then the tail
      using V = typename DsaVec<real>::type;
      constexpr int kN = DsaVec<real>::kN;
      const int nv = N / kN, t0 = blockIdx.x * blockDim.x + threadIdx.x, ts = gridDim.x * blockDim.x;
      // two vectors per thread and round, loads first
      for (int t = t0; t < nv; t += 2 * ts) {
        V pv[2], qv[2], dv[2], xv[2], rv[2], zv[2];
        const bool two = t + ts < nv;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int tg = (g == 0 || two) ? t + g * ts : t;
          pv[g] = reinterpret_cast<const V *>(pn)[tg];
          qv[g] = reinterpret_cast<const V *>(q)[tg];
          dv[g] = reinterpret_cast<const V *>(dinv)[tg];
          xv[g] = reinterpret_cast<const V *>(x)[tg];
          rv[g] = reinterpret_cast<const V *>(r)[tg];
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (g == 1 && !two) break;
          dsa_p2_elem(a, pv[g].x, qv[g].x, xv[g].x, rv[g].x, zv[g].x, dv[g].x, prz, prr);
          dsa_p2_elem(a, pv[g].y, qv[g].y, xv[g].y, rv[g].y, zv[g].y, dv[g].y, prz, prr);
          if constexpr (kN == 4) {
            dsa_p2_elem(a, pv[g].z, qv[g].z, xv[g].z, rv[g].z, zv[g].z, dv[g].z, prz, prr);
            dsa_p2_elem(a, pv[g].w, qv[g].w, xv[g].w, rv[g].w, zv[g].w, dv[g].w, prz, prr);
          }
          const int tg = t + g * ts;
          reinterpret_cast<V *>(x)[tg] = xv[g];
          reinterpret_cast<V *>(r)[tg] = rv[g];
          reinterpret_cast<V *>(z)[tg] = zv[g];
        }
      }
      for (int c = nv * kN + t0; c < N; c += ts) {
        real xc = x[c], rc = r[c], zc;
        dsa_p2_elem(a, pn[c], q[c], xc, rc, zc, dinv[c], prz, prr);
        x[c] = xc;
        r[c] = rc;
        z[c] = zc;
      }
      block_sum2(prz, prr, red);
      if (threadIdx.x == 0) {
        dsa_slot(ctl, i, kDsaRz)[blockIdx.x] = prz;
        dsa_slot(ctl, i, kDsaRr)[blockIdx.x] = prr;
      }
    }
    if (!grid_barrier(ctl.bar, abort_flag)) return false;

    // stop at ||r||_2 <= tol ||b||_2 or the iteration cap; else the next beta
    dsa_sum2(ctl, on, kDsaRz, t0, kDsaRr, t1);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (!on[i]) continue;
      const Inst &I = insts[i];
      if (t1[i] <= I.dsa_tol * I.dsa_tol * bb[i] || k + 1 >= I.dsa_max_iter || !(rz[i] != 0.0)) {
        on[i] = 0;
        if (blockIdx.x == 0) atomicAdd(I.dsa_iters_total, (unsigned long long)(k + 1));
      } else {
        beta[i] = t0[i] / rz[i];
        rz[i] = t0[i];
      }
    }
    __syncthreads();
  }
  return true;
}

}  // namespace dlr
