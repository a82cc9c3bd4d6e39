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
    double v0 = 0, v1 = 0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      v0 += p0[b];
      v1 += p1[b];
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

// z + beta p_old at cell c (the first iteration has p = z)
template <typename real>
__device__ __forceinline__ real dsa_dir(const real *z, const real *po, real beta, bool first, int c) {
  return first ? z[c] : fmadd(beta, po[c], z[c]);
}

// The CG solves of all instances with on[i] (set by the caller: active, DSA
// on, right-hand side nonzero), started from the partials of the scalar-flux
// phase.  sc: 6 x n_inst doubles of shared memory.  Returns false if a grid
// barrier gave up.
template <typename real>
__device__ __noinline__ bool dsa_solve(const Inst *__restrict__ insts, const SiCtl &ctl, int *on,
                                       double *sc, volatile int *abort_flag) {
  __shared__ double red[32];
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
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      const Inst &I = insts[i];
      const int nx = I.nx, ny = I.ny, N = I.N;
      const real *z = as_c<real>(I.dsa_z), *ist = as_c<real>(I.dsa_ist), *dg = as_c<real>(I.dsa_dg);
      const real *po = as_c<real>((k & 1) ? I.dsa_p0 : I.dsa_p1);
      real *pn = as<real>((k & 1) ? I.dsa_p1 : I.dsa_p0);
      real *q = as<real>(I.dsa_q);
      const real b = real(beta[i]);
      const bool first = k == 0;
      const real cx = real(I.dsa_cx), cy = real(I.dsa_cy), kx = real(I.dsa_kx), ky = real(I.dsa_ky);
      double pq = 0;
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int ix = c % nx, iy = c / nx;
        const real uc = dsa_dir(z, po, b, first, c);
        real off = real(0);
        if (ix + 1 < nx) {
          off = fmadd(kx, dsa_dir(z, po, b, first, c + 1), off);
          if (ix + 2 < nx) off = fmadd(cx * ist[c + 1], dsa_dir(z, po, b, first, c + 2), off);
        }
        if (ix >= 1) {
          off = fmadd(kx, dsa_dir(z, po, b, first, c - 1), off);
          if (ix >= 2) off = fmadd(cx * ist[c - 1], dsa_dir(z, po, b, first, c - 2), off);
        }
        if (iy + 1 < ny) {
          off = fmadd(ky, dsa_dir(z, po, b, first, c + nx), off);
          if (iy + 2 < ny) off = fmadd(cy * ist[c + nx], dsa_dir(z, po, b, first, c + 2 * nx), off);
        }
        if (iy >= 1) {
          off = fmadd(ky, dsa_dir(z, po, b, first, c - nx), off);
          if (iy >= 2) off = fmadd(cy * ist[c - nx], dsa_dir(z, po, b, first, c - 2 * nx), off);
        }
        const real Au = fmadd(dg[c], uc, -off);
        pn[c] = uc;
        q[c] = Au;
        pq += (double)uc * (double)Au;
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
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        x[c] = fmadd(a, pn[c], x[c]);
        const real rc = fmadd(-a, q[c], r[c]);
        const real zc = rc * dinv[c];
        r[c] = rc;
        z[c] = zc;
        prz += (double)rc * (double)zc;
        prr += (double)rc * (double)rc;
      }
      prz = block_sum(prz, red);
      prr = block_sum(prr, red);
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
