// k_dense.cu -- per-cell and tall-skinny kernels of the SN-like DLR step
// (Algorithm 1 of Haut et al.):
//   k_coeff_recon  step 1 (Newton-linearised sigma_s, q of Section 2.2) and
//                  step 3 (psi0_j = sum_k X0_k L0_k(Om^(j))), fused with the
//                  fixed source q + psi0_j/(c dt) of the collocation system
//                  and the starting scalar flux gamma^T Psi0
//   k_tsgram       G = sum_c wt_c a_c a_c^T for a tall-skinny matrix (step 5
//                  CholeskyQR Grams of Psi and step 8 Grams of L)
//   k_apply        out = diag(s_out) (diag(s_in) A) T for a small dense T, or
//                  A R^{-1} for a CholeskyQR factor R (forward substitution)
//   k_project      step 6 P = <X, X0> and the step 7 Galerkin operators:
//                  Gram, x/y neighbour Grams, <sigma_t X, X>, <sigma_s X, X>,
//                  <q, X> and the four edge sums (FP64); k_project_tc5 the
//                  same in mixed precision on the tcgen05 tensor cores
//   k_tupdate      step 9 temperature update (Eq. temperature update, Newton
//                  form) with phi = X (L w), fused with the rotation X0 <- X U
// Mixed precision: products and sums over one staging round (at most 128
// rows) in FP32, round sums accumulated in FP64.
#include <algorithm>

#include "dlr_internal.cuh"
#include "tc_core.cuh"

namespace dlr {

constexpr int kTB = 256;      // threads per block of the reduction kernels

// ------------------------------------------------------------------
// step 1 + step 3
// ------------------------------------------------------------------
// grp_mode = 1 (a batch of grouped-sweep instances, mixed precision): the
// fixed sources, sigma_t and the starting sigma_s phi / 4 pi go to the
// skewed layouts of the grouped sweep (each angle in its quadrant's layout;
// sigma_t and sigma_s phi / 4 pi in all four), and block 0 of each instance
// writes the group table (the chosen angles by quadrant, then by index, kGA
// per group); otherwise they go to the plain cell-major arrays.
template <typename real, int RB>
__global__ void __launch_bounds__(256) k_coeff_recon(const Inst *__restrict__ insts, int grp_mode) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (rank_class(I.r) != RB) return;
  __shared__ real C0s[RB * RB];
  __shared__ real gam[RB];
  __shared__ int quadj[RB], grpj[RB], slotj[RB];
  __shared__ int grpq[RB + 4], ngrp;
  const int r = I.r;
  const double *C0 = I.small + I.lay.C0;
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int k = e % RB, j = e / RB;  // C0s[j*RB + k] = C0[k, j]
    C0s[e] = (k < r && j < r) ? real(C0[k + r * j]) : real(0);
  }
  for (int e = threadIdx.x; e < RB; e += blockDim.x) {
    gam[e] = e < r ? real(I.small[I.lay.gamma + e]) : real(0);
    if (grp_mode && e < r) quadj[e] = quad_of(I.ox[I.idx[e]], I.oy[I.idx[e]]);
  }
  __syncthreads();
  if (grp_mode && threadIdx.x == 0) {
    // groups: the chosen angles by quadrant, then by index, kGA per group
    // (every block forms the same table; block 0 stores it)
    const bool store = blockIdx.x == 0;
    int g = 0;
    for (int q = 0; q < 4; ++q) {
      int na = 0;
      for (int j = 0; j < r; ++j) {
        if (quadj[j] != q) continue;
        grpj[j] = g;
        slotj[j] = na;
        grpq[g] = q;
        if (store) {
          int *rec = I.grp_tab + g * kGrpRec;
          rec[0] = q;
          rec[2 + na] = j;
          rec[1] = na + 1;
        }
        if (++na == kGA) { ++g; na = 0; }
      }
      if (na) ++g;
    }
    ngrp = g;
    for (; store && g < I.grp_ng; ++g) {
      int *rec = I.grp_tab + g * kGrpRec;
      rec[0] = 0;
      rec[1] = 0;
      for (int a = 0; a < kGA; ++a) rec[2 + a] = 0;
    }
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= I.N) return;
  // Section 2.2 (Newton linearisation, B = a c T^4 / 4pi)
  const CellCoef cf = cell_coefficients(I, c);
  const double q = cf.q;
  I.B0[c] = cf.B;
  I.D[c] = cf.D;
  const real sig_t = real(cf.sig + I.inv_cdt);
  as<real>(I.sig_t)[c] = sig_t;
  const real ss4 = real(cf.ss / (4.0 * kPi));
  // skewed positions of this cell in the four quadrant layouts (grp_mode)
  size_t go[4] = {0, 0, 0, 0};
  if (grp_mode) {
    const int y = c / I.nx, xx = c - y * I.nx;
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) go[qd] = grp_off(qd, I.nx, I.ny, I.nwin, xx, y);
    // sigma_t beside each group's fixed sources, in the group's quadrant layout
    for (int g = 0; g < ngrp; ++g)
      I.sgk[grp_sgk(I.glay, g, kGA, go[grpq[g]])] = float(sig_t);
  }
  as<real>(I.ss4)[c] = ss4;
  as<real>(I.q)[c] = real(q);
  // psi0 at the chosen angles: Psi0[c, j] = sum_k X0[c, k] C0[k, j]
  const real *X0 = as_c<real>(I.X0);
  real x[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) x[k] = k < r ? X0[(size_t)I.N * k + c] : real(0);
  real *s0 = as<real>(I.s0);
  real phi = real(0);
  const real qr = real(q), icdt = real(I.inv_cdt);
  for (int j = 0; j < r; ++j) {
    real p = real(0);
#pragma unroll
    for (int k = 0; k < RB; ++k) p += x[k] * C0s[j * RB + k];
    if (grp_mode) I.sgk[grp_sgk(I.glay, grpj[j], slotj[j], go[quadj[j]])] = float(qr + icdt * p);
    else s0[(size_t)I.N * j + c] = qr + icdt * p;
    phi += gam[j] * p;
  }
  if (I.aug_x0) {  // augmented step: X0 beside Psi as the input of step 5
    real *xa = as<real>(I.aug_x0);
#pragma unroll
    for (int k = 0; k < RB; ++k)
      if (k < r) xa[(size_t)I.N * k + c] = x[k];
  }
  as<real>(I.phi0)[c] = phi;
  if (grp_mode) {
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) I.spk[(size_t)qd * I.glay + go[qd]] = float(ss4 * phi);
  } else {
    as<real>(I.sphi)[c] = ss4 * phi;
  }
}

// ------------------------------------------------------------------
// tall-skinny Gram, one thread-block cluster per slice of rows (r <= 32)
// ------------------------------------------------------------------
// A is m x r; layout 0: column-major A[row + lda*i]; layout 1: rows of r
// contiguous A[i + r*row].  wt: per-row weight or nullptr.  The CTAs of a
// job split the rows evenly; each stages GR rows per round in shared memory
// (column-major, the next round prefetched into registers while the current
// one is multiplied) and every thread accumulates a 4 x 4 tile of G over the
// rows of its group.  FP32 tiles are added to FP64 accumulators after every
// round.  The CTA partial is summed over the cluster through distributed
// shared memory (fixed order); cluster c writes its r x r sum (FP64,
// column-major) to out + c*r*r.
template <typename real> struct GramCfg;
template <> struct GramCfg<float> { static constexpr int GR = 128; };
template <> struct GramCfg<double> { static constexpr int GR = 64; };

template <typename real>
constexpr int gram_smem_bytes() {
  constexpr int GR = GramCfg<real>::GR;
  constexpr int tiles = (2 * 32 * (GR + 4) + GR) * (int)sizeof(real);
  constexpr int red = (kTB * 16 + 32 * 32) * 8;
  return tiles > red ? tiles : red;
}

template <typename real, int LAY>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kTB)
k_tsgram(const GramJob *__restrict__ jobs) {
  pdl_wait();
  pdl_trigger();
  constexpr int GR = GramCfg<real>::GR, LD = GR + 4;
  constexpr int PF = GR * 32 / kTB;  // prefetched elements per thread and matrix
  const GramJob J = jobs[blockIdx.y];
  // nblocks is a multiple of the cluster size and run_if is per job, so
  // whole clusters leave together
  if ((int)blockIdx.x >= J.nblocks || (J.run_if && *J.run_if == 0)) return;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ __align__(32) unsigned char raw[gram_smem_bytes<real>()];
  real *As = reinterpret_cast<real *>(raw);
  real *Bs = As + 32 * LD;
  real *ws = Bs + 32 * LD;
  const int r = J.r, t = threadIdx.x;
  const int side = (r + 3) >> 2, ntile = side * side;
  const int ngroup = kTB / ntile;
  const int grp = t / ntile, tt = t - grp * ntile;
  const int ti = 4 * (tt % side), tj = 4 * (tt / side);
  const bool cross = J.B != nullptr;
  // a symmetric Gram needs the tiles on and above the diagonal only
  const bool own = grp < ngroup && (cross || tj >= ti);
  const real *A = as_c<real>(J.A), *Bm = as_c<real>(J.B);
  const int per = (J.m + J.nblocks - 1) / J.nblocks;
  const int row0 = min(J.m, (int)blockIdx.x * per), row1 = min(J.m, row0 + per);
  const int nround = (row1 - row0 + GR - 1) / GR;
  // (row, column) of the elements this thread stages, fixed for all rounds
  int erow[PF], ecol[PF];
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    const int e = t + kTB * k;
    erow[k] = LAY == 0 ? e % GR : e / r;
    ecol[k] = LAY == 0 ? e / GR : e % r;
    if (erow[k] >= GR || ecol[k] >= r) ecol[k] = 32;  // not staged
  }
  // rounds per FP32 partial: about 64 rows per thread before the FP64 add
  const int flush_every = max(1, 64 * ngroup / GR);
  // The prefetch issues plain loads from clamped (always valid) addresses
  // and keeps the raw values: no arithmetic touches them until they are
  // staged, so the loads stay in flight during the products.
  real pa[PF], pbv[PF];
  double pw = 0.0;
  auto prefetch = [&](int rd) {
    const int base = row0 + rd * GR;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int row = min(base + erow[k], row1 - 1), i = min(ecol[k], r - 1);
      const size_t at = LAY == 0 ? (size_t)J.lda * i + row : (size_t)r * row + i;
      pa[k] = A[at];
      if (cross) pbv[k] = Bm[(size_t)J.ldb * i + row];
    }
    if (t < GR && J.wt) pw = J.wt[min(base + t, row1 - 1)];
  };
  real s[16];
  double acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) { s[e] = real(0); acc[e] = 0.0; }
  if (nround > 0) prefetch(0);
  for (int rd = 0; rd < nround; ++rd) {
    __syncthreads();  // the previous round's products are done
    const int base = row0 + rd * GR;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int rr = erow[k], i = ecol[k];
      if (i < 32) {
        const bool ok = base + rr < row1;
        As[i * LD + rr] = ok ? pa[k] : real(0);
        if (cross) Bs[i * LD + rr] = ok ? pbv[k] : real(0);
      }
    }
    if (t < GR) {
      double w = base + t < row1 ? (J.wt ? pw : 1.0) : 0.0;
      if (J.sqrt_wt) w = sqrt(w);
      ws[t] = real(w);
    }
    __syncthreads();
    if (rd + 1 < nround) prefetch(rd + 1);  // in flight during the products below
    if (own) {
      const real *Bsrc = cross ? Bs : As;
      const int nq = (min(GR, row1 - row0 - rd * GR) + 3) >> 2;  // quads holding rows
      for (int q = grp; q < nq; q += ngroup) {
        Quad<real> a[4], b[4];
        const Quad<real> w = *reinterpret_cast<const Quad<real> *>(ws + 4 * q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          a[k] = *reinterpret_cast<const Quad<real> *>(As + (ti + k) * LD + 4 * q);
          b[k] = *reinterpret_cast<const Quad<real> *>(Bsrc + (tj + k) * LD + 4 * q);
#pragma unroll
          for (int m = 0; m < 4; ++m) a[k].v[m] *= w.v[m];
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < 4; ++m) s[kk * 4 + k] += a[kk].v[m] * b[k].v[m];
      }
      if (sizeof(real) == 4 && ((rd + 1) % flush_every == 0 || rd + 1 == nround)) {
#pragma unroll
        for (int e = 0; e < 16; ++e) { acc[e] += (double)s[e]; s[e] = real(0); }
      }
    }
  }
  if (sizeof(real) != 4) {
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = (double)s[e];
  }
  // groups -> CTA partial (fixed order), tile entries of the lower triangle
  // of a symmetric Gram mirrored from the upper one
  __syncthreads();
  double *buf = reinterpret_cast<double *>(raw);
  double *part_s = buf + kTB * 16;
  if (grp < ngroup) {
#pragma unroll
    for (int e = 0; e < 16; ++e) buf[t * 16 + e] = acc[e];
  }
  __syncthreads();
  for (int e = t; e < r * r; e += kTB) {
    int i = e % r, j = e / r;
    if (!cross && i > j) { const int x = i; i = j; j = x; }
    const int tl = (i >> 2) + side * (j >> 2), comp = (i & 3) * 4 + (j & 3);
    double v = 0.0;
    for (int g = 0; g < ngroup; ++g) v += buf[(g * ntile + tl) * 16 + comp];
    part_s[e] = v;
  }
  cluster.sync();
  // this CTA's share of the cluster sum, CTA partials added in rank order
  const int rank = (int)cluster.block_rank();
  const int rr2 = r * r, share = (rr2 + kCl - 1) / kCl;
  double *out = J.out + (size_t)(blockIdx.x / kCl) * rr2;
  for (int e = rank * share + t; e < min(rr2, (rank + 1) * share); e += kTB) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < kCl; ++q) v += cluster.map_shared_rank(part_s, q)[e];
    out[e] = v;
  }
  cluster.sync();  // peers' shared memory stays valid until every read is done
}

// ------------------------------------------------------------------
// orthonormal completion: dependent columns replaced by pseudo-random ones
// ------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(256) k_fill(const FillJob *__restrict__ jobs) {
  pdl_wait();
  pdl_trigger();
  const FillJob J = jobs[blockIdx.y];
  const int nfill = J.flag[1];
  if (!J.src && nfill == 0) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= J.m) return;
  real *A = as<real>(J.A);
  const real *S = as_c<real>(J.src);
  for (int j = 0; j < J.r; ++j) {
    const size_t at = J.layout == 0 ? (size_t)J.lda * j + row : (size_t)J.r * row + j;
    if (nfill && J.flag[2 + j]) A[at] = real(hash_uniform(((unsigned long long)j << 40) ^ (unsigned long long)row));
    else if (S) A[at] = S[at];
  }
}

// ------------------------------------------------------------------
// out[row, :] = s_out[row] * (s_in[row] * A[row, :]) * T    (T is r x r)
// ------------------------------------------------------------------

template <typename rin, typename rout, int RB>
__global__ void __launch_bounds__(128) k_apply(const ApplyJob *__restrict__ jobs) {
  pdl_wait();
  pdl_trigger();
  const ApplyJob J = jobs[blockIdx.y];
  if (rank_class(J.r) != RB || (J.run_if && *J.run_if == 0)) return;
  __shared__ rout Ts[RB * RB];
  __shared__ rout dg[RB];
  const int r = J.r;
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int i = e % RB, j = e / RB;
    Ts[e] = (i < r && j < r) ? rout(J.T[i + r * j]) : rout(i == j && J.tri ? 1 : 0);
  }
  if (J.tri)
    for (int j = threadIdx.x; j < RB; j += blockDim.x) dg[j] = j < r ? rout(1.0 / J.T[j + r * j]) : rout(1);
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= J.m) return;
  const rin *A = as_c<rin>(J.A);
  rout a[RB];
  rout sc = rout(1);
  if (J.s_in) sc = rout(J.sq_in ? sqrt(J.s_in[row]) : J.s_in[row]);
#pragma unroll
  for (int i = 0; i < RB; ++i)
    a[i] = i < r ? sc * rout(J.in_layout == 0 ? A[(size_t)J.lda * i + row] : A[(size_t)r * row + i])
                 : rout(0);
  rout so = rout(1);
  if (J.s_out) so = rout(J.inv_sq_out ? 1.0 / sqrt(J.s_out[row]) : J.s_out[row]);
  rout *O = as<rout>(J.out);
  if (J.tri) {
    // x R = a by forward substitution (R upper triangular), x in place of a
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      rout v = a[j];
#pragma unroll
      for (int i = 0; i < j; ++i) v -= a[i] * Ts[j * RB + i];
      a[j] = v * dg[j];
    }
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if (j < r) O[(size_t)J.ldo * j + row] = so * a[j];
    return;
  }
  for (int j = 0; j < r; ++j) {
    rout v = rout(0);
#pragma unroll
    for (int i = 0; i < RB; ++i) v += a[i] * Ts[j * RB + i];
    O[(size_t)J.ldo * j + row] = so * v;
  }
}

// ------------------------------------------------------------------
// step 6 / step 7 projections, one thread-block cluster per slice of cells.
// Per-cluster partial (FP64) layout, r x r column-major each: G, Nx, Ny,
// Mt, Ms, P, then vec[5r]: qh, bL, bR, bB, bT.
//   G_ij  = sum_c X_ci X_cj            Mt_ij = sum_c sig_t X_ci X_cj
//   Ms_ij = sum_c sigma_s X_ci X_cj    P_ij  = sum_c X_ci X0_cj
//   Nx_ij = sum_{ix>=1} X_ci X_{c-1,j} Ny_ij = sum_{iy>=1} X_ci X_{c-nx,j}
//   qh_i  = sum_c q_c X_ci             bL_i  = sum_{ix=0} X_ci, ...
// (all without the h^2 factor, applied in the reduction).  Threads come in
// two kinds over 4 x 2 tiles of the r x r outputs: kind 0 accumulates G,
// Mt, Ms (and qh), kind 1 Nx, Ny, P (and the four edge sums).  Staging,
// prefetch, FP32-round/FP64-total accumulation and the cluster sum are as in
// k_tsgram.
// ------------------------------------------------------------------
template <typename real> struct ProjCfg;
template <> struct ProjCfg<float> { static constexpr int GP = 64; };
template <> struct ProjCfg<double> { static constexpr int GP = 32; };

template <typename real>
constexpr int proj_tile_bytes() {
  return (4 * 32 * (ProjCfg<real>::GP + 4) + 9 * ProjCfg<real>::GP) * (int)sizeof(real);
}
inline int proj_smem_bytes(int r, int rs) {
  const int tiles = rs == 4 ? proj_tile_bytes<float>() : proj_tile_bytes<double>();
  const int red = (kTB * 16 + proj_count(r)) * 8;
  return tiles > red ? tiles : red;
}

template <typename real>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kTB)
k_project(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  constexpr int GP = ProjCfg<real>::GP, LD = GP + 4;
  constexpr int PF = GP * 32 / kTB;
  const Inst &I = insts[blockIdx.y];
  const int nblk = I.partial_blocks;
  if ((int)blockIdx.x >= nblk) return;  // whole clusters
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(32) unsigned char dyn[];
  real *Xs = reinterpret_cast<real *>(dyn);
  real *XLs = Xs + 32 * LD, *XBs = XLs + 32 * LD, *X0s = XBs + 32 * LD;
  real *vs = X0s + 32 * LD;  // 9 x GP: sig_t, sigma_s, q, mL, mB, eL, eR, eB, eT
  const int r = I.r, N = I.N, nx = I.nx, ny = I.ny, t = threadIdx.x;
  const int s4 = (r + 3) >> 2, s2 = (r + 1) >> 1, ntile = s4 * s2;
  const int gsz = 2 * ntile, ngroup = kTB / gsz;
  const int grp = t / gsz, l = t - grp * gsz;
  const int kind = l / ntile, tt = l - kind * ntile;
  const int ti = 4 * (tt % s4), tj = 2 * (tt / s4);
  const bool own = grp < ngroup;
  const bool vec_owner = own && tj == 0;
  const real *__restrict__ X = as_c<real>(I.X);
  const real *__restrict__ X0 = as_c<real>(I.X0);
  const real *__restrict__ sig_t = as_c<real>(I.sig_t);
  const real *__restrict__ ss4 = as_c<real>(I.ss4);
  const real *__restrict__ qv = as_c<real>(I.q);
  double *const partials = I.partials;
  const int per = (N + nblk - 1) / nblk;
  const int c0 = min(N, (int)blockIdx.x * per), c1 = min(N, c0 + per);
  const int nround = (c1 - c0 + GP - 1) / GP;
  // raw loads from clamped addresses (masks applied when staging), as in
  // k_tsgram; the left and lower neighbours of cells on the first column or
  // row are masked by mL and mB in the products
  real px[PF], pl[PF], pd[PF], p0[PF], pv[3];
  auto prefetch = [&](int rd) {
    const int base = c0 + rd * GP;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int e = t + kTB * k, rr = e % GP, i = min(e / GP, r - 1);
      const int c = min(base + rr, c1 - 1);
      const size_t col = (size_t)N * i;
      px[k] = X[col + c];
      pl[k] = X[col + max(c - 1, 0)];
      pd[k] = X[col + max(c - nx, 0)];
      p0[k] = X0[col + c];
    }
    if (t < GP) {
      const int c = min(base + t, c1 - 1);
      pv[0] = sig_t[c];
      pv[1] = ss4[c];
      pv[2] = qv[c];
    }
  };
  // three levels of sums in the working precision (a round, up to eight
  // rounds, all rounds), converted to FP64 once at the end: the FP64 pipe
  // stays out of the loop, and no FP32 sum runs over more than about 64
  // terms
  real sm[24], sv[16], m2[24], v2[16], m3[24], v3[16];
  double am[24], av[16];
#pragma unroll
  for (int e = 0; e < 24; ++e) { sm[e] = real(0); m2[e] = real(0); m3[e] = real(0); }
#pragma unroll
  for (int e = 0; e < 16; ++e) { sv[e] = real(0); v2[e] = real(0); v3[e] = real(0); }
  if (nround > 0) prefetch(0);
  for (int rd = 0; rd < nround; ++rd) {
    __syncthreads();
    const int base = c0 + rd * GP;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int e = t + kTB * k, rr = e % GP, i = e / GP;
      if (i < r) {
        const bool ok = base + rr < c1;
        Xs[i * LD + rr] = ok ? px[k] : real(0);
        XLs[i * LD + rr] = ok ? pl[k] : real(0);
        XBs[i * LD + rr] = ok ? pd[k] : real(0);
        X0s[i * LD + rr] = ok ? p0[k] : real(0);
      }
    }
    if (t < GP) {
      const int c = base + t;
      const bool ok = c < c1;
      const int pix = ok ? c % nx : -1, piy = ok ? c / nx : -1;
      vs[0 * GP + t] = ok ? pv[0] : real(0);
      vs[1 * GP + t] = ok ? pv[1] * real(4.0 * kPi) : real(0);
      vs[2 * GP + t] = ok ? pv[2] : real(0);
      vs[3 * GP + t] = real(ok && pix >= 1);
      vs[4 * GP + t] = real(ok && piy >= 1);
      vs[5 * GP + t] = real(ok && pix == 0);
      vs[6 * GP + t] = real(ok && pix == nx - 1);
      vs[7 * GP + t] = real(ok && piy == 0);
      vs[8 * GP + t] = real(ok && piy == ny - 1);
    }
    __syncthreads();
    if (rd + 1 < nround) prefetch(rd + 1);
    if (own) {
      const int nq = (min(GP, c1 - c0 - rd * GP) + 3) >> 2;  // quads holding cells
      for (int q = grp; q < nq; q += ngroup) {
        Quad<real> a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = *reinterpret_cast<const Quad<real> *>(Xs + (ti + k) * LD + 4 * q);
        if (kind == 0) {
          Quad<real> b[2];
#pragma unroll
          for (int k = 0; k < 2; ++k) b[k] = *reinterpret_cast<const Quad<real> *>(Xs + (tj + k) * LD + 4 * q);
          const Quad<real> st = *reinterpret_cast<const Quad<real> *>(vs + 4 * q);
          const Quad<real> ss = *reinterpret_cast<const Quad<real> *>(vs + GP + 4 * q);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
              for (int m = 0; m < 4; ++m) {
                const real p = a[kk].v[m] * b[k].v[m];
                sm[kk * 2 + k] += p;
                sm[8 + kk * 2 + k] += st.v[m] * p;
                sm[16 + kk * 2 + k] += ss.v[m] * p;
              }
          if (vec_owner) {
            const Quad<real> qq = *reinterpret_cast<const Quad<real> *>(vs + 2 * GP + 4 * q);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
#pragma unroll
              for (int m = 0; m < 4; ++m) sv[kk] += qq.v[m] * a[kk].v[m];
          }
        } else {
          Quad<real> bl[2], bd[2], b0[2];
          const Quad<real> ml = *reinterpret_cast<const Quad<real> *>(vs + 3 * GP + 4 * q);
          const Quad<real> mb = *reinterpret_cast<const Quad<real> *>(vs + 4 * GP + 4 * q);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            bl[k] = *reinterpret_cast<const Quad<real> *>(XLs + (tj + k) * LD + 4 * q);
            bd[k] = *reinterpret_cast<const Quad<real> *>(XBs + (tj + k) * LD + 4 * q);
            b0[k] = *reinterpret_cast<const Quad<real> *>(X0s + (tj + k) * LD + 4 * q);
#pragma unroll
            for (int m = 0; m < 4; ++m) { bl[k].v[m] *= ml.v[m]; bd[k].v[m] *= mb.v[m]; }
          }
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
              for (int m = 0; m < 4; ++m) {
                sm[kk * 2 + k] += a[kk].v[m] * bl[k].v[m];
                sm[8 + kk * 2 + k] += a[kk].v[m] * bd[k].v[m];
                sm[16 + kk * 2 + k] += a[kk].v[m] * b0[k].v[m];
              }
          if (vec_owner) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const Quad<real> ev = *reinterpret_cast<const Quad<real> *>(vs + (5 + v) * GP + 4 * q);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                for (int m = 0; m < 4; ++m) sv[v * 4 + kk] += ev.v[m] * a[kk].v[m];
            }
          }
        }
      }
      if (sizeof(real) == 4) {
#pragma unroll
        for (int e = 0; e < 24; ++e) { m2[e] += sm[e]; sm[e] = real(0); }
#pragma unroll
        for (int e = 0; e < 16; ++e) { v2[e] += sv[e]; sv[e] = real(0); }
        if ((rd + 1) % 8 == 0) {
#pragma unroll
          for (int e = 0; e < 24; ++e) { m3[e] += m2[e]; m2[e] = real(0); }
#pragma unroll
          for (int e = 0; e < 16; ++e) { v3[e] += v2[e]; v2[e] = real(0); }
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 24; ++e) am[e] = (double)sm[e] + ((double)m2[e] + (double)m3[e]);
#pragma unroll
  for (int e = 0; e < 16; ++e) av[e] = (double)sv[e] + ((double)v2[e] + (double)v3[e]);
  // groups -> CTA partial in a fixed order, one output slot at a time
  double *buf = reinterpret_cast<double *>(dyn);
  double *part_s = buf + kTB * 16;
  const int rr2 = r * r;
  for (int slot = 0; slot < 3; ++slot) {
    __syncthreads();
    if (own) {
#pragma unroll
      for (int e = 0; e < 8; ++e) buf[t * 8 + e] = am[slot * 8 + e];
    }
    __syncthreads();
    for (int e = t; e < 2 * rr2; e += kTB) {
      const int kd = e / rr2, ij = e - kd * rr2, i = ij % r, j = ij / r;
      const int lt = kd * ntile + (i >> 2) + s4 * (j >> 1), comp = (i & 3) * 2 + (j & 1);
      double v = 0.0;
      for (int g = 0; g < ngroup; ++g) v += buf[(g * gsz + lt) * 8 + comp];
      // kind 0 holds G, Mt, Ms (blocks 0, 3, 4); kind 1 Nx, Ny, P (1, 2, 5)
      const int mat = kd == 0 ? (slot == 0 ? 0 : slot + 2) : (slot == 2 ? 5 : slot + 1);
      part_s[mat * rr2 + ij] = v;
    }
  }
  __syncthreads();
  if (own) {
#pragma unroll
    for (int e = 0; e < 16; ++e) buf[t * 16 + e] = av[e];
  }
  __syncthreads();
  for (int e = t; e < 5 * r; e += kTB) {
    const int v = e / r, i = e - v * r;
    const int lt = (v == 0 ? 0 : ntile) + (i >> 2), comp = (v == 0 ? 0 : (v - 1) * 4) + (i & 3);
    double x = 0.0;
    for (int g = 0; g < ngroup; ++g) x += buf[(g * gsz + lt) * 16 + comp];
    part_s[6 * rr2 + e] = x;
  }
  cluster.sync();
  const int rank = (int)cluster.block_rank();
  const int cnt = proj_count(r), share = (cnt + kCl - 1) / kCl;
  double *out = partials + (size_t)(blockIdx.x / kCl) * cnt;
  for (int e = rank * share + t; e < min(cnt, (rank + 1) * share); e += kTB) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < kCl; ++q) v += cluster.map_shared_rank(part_s, q)[e];
    out[e] = v;
  }
  cluster.sync();
}

// cp.async helpers (4- and 16-byte copies, zero-filled past src_bytes)
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------
// step 6 / step 7 projections on the fifth-generation tensor cores
// (tcgen05; tc_core.cuh), mixed precision.  The same sums as
// k_project<float> (G, Nx, Ny, Mt, Ms, P and the vector sums), written as
// one product per CTA slice of cells, D^T = B^T X with the operand columns
//   B = [X, X_L, X_B, sig_t X, (sigma_s / 4 pi) X, X0, q, e_L, e_R, e_B, e_T]
// (X_L(c) = X(c - 1) on cells with ix >= 1, X_B(c) = X(c - nx) on cells with
// iy >= 1, zero elsewhere; e_* the indicators of the four edges' cells).
// Per cell this is 6 r^2 + 5 r multiply-adds on 8 r + 12 bytes, too dense
// for the FP32 pipe to keep up with HBM.  The 6 r + 5 operand columns are
// the M side (128 or 256 rows, two M = 128 accumulators at rank
// 32) and the r columns of X as the N side (16 or 32), the FP32
// accumulators in tensor memory.  16 producer warps stage cells in chunks of
// 32 (4 k-steps) into three raw stages (cp.async; 16-byte copies when N and
// nx are multiples of 4, else 4-byte ones; zero-filled past the slice, past
// rank r and where the shifted neighbour does not exist) and form
// the operands of a chunk (scaled, shifted, split into TF32 parts) in the
// tensor core's layout in one of two operand buffers, each thread owning
// one operand row for the whole kernel; a 17th warp issues the chunk's 24
// MMAs (3 split products per k-step and half) once the producers have
// arrived on the buffer's "full" mbarrier and commits them to its "empty"
// mbarrier, which the producers wait on before refilling it.  TF32 split
// products (tc_core.cuh): each operand value x is stored as hi = x rounded
// to TF32 and lo = x - hi, a product summed as hi lo + lo hi + hi hi.
// Producers meet on one named barrier per chunk; the MMA warp never joins
// it.  Pairs
// of chunks (64 cells) accumulate alternately in two sets of accumulators;
// a pair's set is read into FP32 registers (the owner of D row m, lane
// m % 128 of half m / 128) once its products have completed; FP32 sums per
// 8 pairs and per slice, FP64 once, one partial per CTA (at most one CTA
// per SM and no cluster, so every SM takes a slice).  Every mbarrier wait
// is bounded; a wait that runs out marks the instance DLR_ETIMEOUT.
// ------------------------------------------------------------------
constexpr int kQP = 512;          // producer threads (16 warps)
constexpr int kQT = kQP + 32;     // and the MMA warp
constexpr int kQKC = 32;          // cells per chunk (4 k-steps)
constexpr int kQLD = kQKC + 4;    // raw stage column stride: 4 cells of halo in front
constexpr int kQS = 3;            // raw stages
constexpr uint64_t kQWaitNs = 2000000000ull;

template <int RB> struct Q5 {
  static constexpr int H = RB == 32 ? 2 : 1;          // M = 128 halves
  static constexpr int M = 128 * H;                   // operand rows (6 RB + 5 used)
  static constexpr int N = RB < 16 ? 16 : RB;         // X columns (padded to 16)
  static constexpr int RAW = 3 * RB * kQLD + 9 * kQKC;  // floats of a raw stage
  static constexpr int OPA = M * kQKC;                // floats of one A copy (hi or lo)
  static constexpr int OPB = N * kQKC;
  static constexpr int BUF = 2 * OPA + 2 * OPB;       // floats of one operand buffer
  static constexpr int NCOL = 2 * H * N <= 32 ? 32 : 2 * H * N <= 64 ? 64 : 128;  // two accumulator sets
  // operand-forming threads: A rows padded to whole warps, JA (JB) groups
  // of 4 cells in parallel per row
  static constexpr int MRP = (6 * RB + 5 + 31) / 32 * 32;
  static constexpr int JA = RB == 32 ? 2 : RB == 16 ? 2 : 4;
  static constexpr int JB = RB == 32 ? 2 : 8;
  static_assert(MRP * JA + RB * JB <= kQP, "operand roles exceed the producers");
  static constexpr int OFF_BUF = ((kQS * RAW * 4 + 1023) / 1024) * 1024;
  static constexpr int OFF_BAR = OFF_BUF + 2 * BUF * 4;  // full[2], empty[2]
  // the readers' per-slice FP32 sums: N values of 128 H threads, column-major
  static constexpr int OFF_ACC = OFF_BAR + 32;
  static constexpr int SMEM = OFF_ACC + N * 128 * H * 4;
};

__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"r"(kQP) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(tc::saddr(m)) : "memory");
}

template <int RB>
__global__ void __launch_bounds__(kQT, 1) k_project_tc5(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  using C = Q5<RB>;
  const Inst &I = insts[blockIdx.y];
  if (rank_class(I.r) != RB) return;
  const int nblk = I.partial_blocks;
  if ((int)blockIdx.x >= nblk) return;
  extern __shared__ __align__(1024) unsigned char dyn5[];
  float *raw = reinterpret_cast<float *>(dyn5);
  unsigned char *opbuf = dyn5 + C::OFF_BUF;
  uint64_t *full = reinterpret_cast<uint64_t *>(dyn5 + C::OFF_BAR), *empty = full + 2;
  __shared__ uint32_t tslot;
  __shared__ int bad;
  const int r = I.r, N = I.N, nx = I.nx, ny = I.ny, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const float *__restrict__ X = as_c<float>(I.X);
  const float *__restrict__ X0 = as_c<float>(I.X0);
  const float *__restrict__ sig_t = as_c<float>(I.sig_t);
  const float *__restrict__ ss4 = as_c<float>(I.ss4);
  const float *__restrict__ qv = as_c<float>(I.q);
  const bool vec = (N & 3) == 0 && (nx & 3) == 0 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(X0) & 15) == 0) && ((reinterpret_cast<uintptr_t>(sig_t) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(ss4) & 15) == 0) && ((reinterpret_cast<uintptr_t>(qv) & 15) == 0);
  const int per = ((N + nblk - 1) / nblk + 3) & ~3;
  const int c0 = min(N, (int)blockIdx.x * per), c1 = min(N, c0 + per);
  const int nchunk = (c1 - c0 + kQKC - 1) / kQKC;

  // the operand buffers' padding rows stay zero throughout
  for (int e = t; e < C::BUF / 2; e += kQT)
    reinterpret_cast<float4 *>(opbuf)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (t == 0) {
    tc::mbar_init(full, kQP / 32);
    tc::mbar_init(full + 1, kQP / 32);
    tc::mbar_init(empty, 1);
    tc::mbar_init(empty + 1, 1);
    bad = 0;
  }
  if (w == 0) tc::alloc(&tslot, C::NCOL);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(128, C::N);

  // this thread's FP32 sums of the accumulator rows it reads: per 8 pairs
  // in registers, per slice in shared memory (acc3[e * 128 H + t])
  float acc2[C::N];
#pragma unroll
  for (int e = 0; e < C::N; ++e) acc2[e] = 0.f;
  const bool reader = w < 4 * C::H;
  float *acc3 = reinterpret_cast<float *>(dyn5 + C::OFF_ACC);
  constexpr int NR = 128 * C::H;
  if (reader)
#pragma unroll
    for (int e = 0; e < C::N; ++e) acc3[e * NR + t] = 0.f;

  if (w == kQP / 32) {
    // the MMA warp
    if (lane == 0) {
      unsigned fpar[2] = {0u, 0u};
      for (int ch = 0; ch < nchunk; ++ch) {
        const int b = ch & 1, set = (ch >> 1) & 1;
        if (!tc::mbar_wait(full + b, fpar[b], kQWaitNs)) break;  // the producers gave up
        fpar[b] ^= 1u;
        tc::fence_after_sync();
        const unsigned char *Ah = opbuf + (size_t)b * C::BUF * 4, *Al = Ah + C::OPA * 4;
        const unsigned char *Bh = Al + C::OPA * 4, *Bl = Bh + C::OPB * 4;
#pragma unroll
        for (int s = 0; s < kQKC / 8; ++s)
#pragma unroll
          for (int hf = 0; hf < C::H; ++hf) {
            const uint32_t d = tmem + (uint32_t)(set * C::H * C::N + hf * C::N);
            const uint32_t ao = (uint32_t)(s * C::M * 32 + hf * 4096), bo = (uint32_t)(s * C::N * 32);
            tc::mma(d, tc::smem_desc(tc::saddr(Ah + ao)), tc::smem_desc(tc::saddr(Bl + bo)), idesc,
                    !((ch & 1) == 0 && s == 0));
            tc::mma(d, tc::smem_desc(tc::saddr(Al + ao)), tc::smem_desc(tc::saddr(Bh + bo)), idesc, true);
            tc::mma(d, tc::smem_desc(tc::saddr(Ah + ao)), tc::smem_desc(tc::saddr(Bh + bo)), idesc, true);
          }
        tc::commit(empty + b);
      }
    }
    __syncwarp();
  } else {
    // the producers
    auto issue = [&](int ch) {
      float *S = raw + (ch % kQS) * C::RAW;
      const int base = c0 + ch * kQKC;
      if (vec) {
        constexpr int QX = kQLD / 4;
        for (int e = t; e < RB * QX; e += kQP) {
          const int i = e / QX, h = 4 * (e - i * QX), c = base - 4 + h;
          const bool ok = i < r && c >= 0 && c < c1;
          cp_async16(S + i * kQLD + h, ok ? X + (size_t)N * i + c : X, ok ? 16 : 0);
        }
        constexpr int QK = kQKC / 4;
        for (int e = t; e < RB * QK; e += kQP) {
          const int i = e / QK, k = 4 * (e - i * QK), c = base + k;
          const bool okc = i < r && c < c1, okb = okc && c >= nx;
          cp_async16(S + (RB + i) * kQLD + 4 + k, okb ? X + (size_t)N * i + (c - nx) : X, okb ? 16 : 0);
          cp_async16(S + (2 * RB + i) * kQLD + 4 + k, okc ? X0 + (size_t)N * i + c : X0, okc ? 16 : 0);
        }
        if (t < 3 * QK) {
          const int row = t / QK, k = 4 * (t - row * QK), c = base + k;
          const float *src = row == 0 ? sig_t : row == 1 ? ss4 : qv;
          cp_async16(S + 3 * RB * kQLD + row * kQKC + k, c < c1 ? src + c : src, c < c1 ? 16 : 0);
        }
      } else {
        for (int e = t; e < RB * (kQKC + 1); e += kQP) {
          const int i = e / (kQKC + 1), h = e - i * (kQKC + 1) + 3, c = base - 4 + h;
          const bool ok = i < r && c >= 0 && c < c1;
          cp_async4(S + i * kQLD + h, ok ? X + (size_t)N * i + c : X, ok ? 4 : 0);
        }
        for (int e = t; e < RB * kQKC; e += kQP) {
          const int i = e / kQKC, k = e - i * kQKC, c = base + k;
          const bool okc = i < r && c < c1, okb = okc && c >= nx;
          cp_async4(S + (RB + i) * kQLD + 4 + k, okb ? X + (size_t)N * i + (c - nx) : X, okb ? 4 : 0);
          cp_async4(S + (2 * RB + i) * kQLD + 4 + k, okc ? X0 + (size_t)N * i + c : X0, okc ? 4 : 0);
        }
        if (t < 3 * kQKC) {
          const int row = t / kQKC, k = t - row * kQKC, c = base + k;
          const float *src = row == 0 ? sig_t : row == 1 ? ss4 : qv;
          cp_async4(S + 3 * RB * kQLD + row * kQKC + k, c < c1 ? src + c : src, c < c1 ? 4 : 0);
        }
      }
      if (t >= kQP - kQKC) {  // masks: rows 3 .. 8 of the per-cell block
        float *V = S + 3 * RB * kQLD;
        const int k = t - (kQP - kQKC), c = base + k;
        const bool ok = c < c1;
        const int iy = ok ? c / nx : 0, ix = ok ? c - iy * nx : 0;
        V[3 * kQKC + k] = (ok && ix >= 1) ? 1.f : 0.f;
        V[4 * kQKC + k] = (ok && ix == 0) ? 1.f : 0.f;
        V[5 * kQKC + k] = (ok && ix == nx - 1) ? 1.f : 0.f;
        V[6 * kQKC + k] = (ok && iy == 0) ? 1.f : 0.f;
        V[7 * kQKC + k] = (ok && iy == ny - 1) ? 1.f : 0.f;
        V[8 * kQKC + k] = 1.f;
      }
    };
    // operand roles (fixed for the kernel): A: thread t < MRP JA owns row
    // m = t % MRP and the groups t / MRP + JA p; B: the next RB JB threads
    // own X column n and the groups (t - MRP JA) / RB + JB p
    constexpr int MRP = C::MRP;
    const bool arole = t < MRP * C::JA && (t % MRP) < 6 * RB + 5;
    const bool brole = t >= MRP * C::JA && t < MRP * C::JA + RB * C::JB;
    int ajg = 0, arow_s = 0, arow_c = 0, bjg = 0, brow_c = 0;
    uint32_t arow_o = 0, brow_o = 0;
    bool avec = false, ashift = false;
    if (t < MRP * C::JA) {
      const int m = t % MRP;
      ajg = t / MRP;
      arow_o = (uint32_t)((m >> 3) * 256 + (m & 7) * 16);
      if (m < 6 * RB) {
        const int mat = m / RB, col = m - mat * RB;
        const int srow = mat == 1 ? 3 : mat == 3 ? 0 : mat == 4 ? 1 : 8;  // mL, sig_t, sigma_s/4pi, 1
        arow_s = 3 * RB * kQLD + srow * kQKC;
        arow_c = (mat == 2 ? RB + col : mat == 5 ? 2 * RB + col : col) * kQLD + 4;
        ashift = mat == 1;
      } else {
        const int v = m - 6 * RB;  // q, eL, eR, eB, eT
        arow_s = 3 * RB * kQLD + (v == 0 ? 2 : v + 3) * kQKC;
        avec = true;
      }
    } else if (brole) {
      const int tb = t - MRP * C::JA, n = tb % RB;
      bjg = tb / RB;
      brow_c = n * kQLD + 4;
      brow_o = (uint32_t)((n >> 3) * 256 + (n & 7) * 16);
    }
    int nflush = 0;
    auto flush_set = [&](int set) {  // the set's products have completed
      tc::fence_after_sync();
      if (reader) {
        const uint32_t ta =
            tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(set * C::H * C::N + (w >> 2) * C::N);
        if (C::N == 32) {
          float v[32];
          tc::ld32(ta, v);
#pragma unroll
          for (int e = 0; e < C::N; ++e) acc2[e] += v[e % 32];
        } else {
          float v[16];
          tc::ld16(ta, v);
#pragma unroll
          for (int e = 0; e < C::N; ++e) acc2[e] += v[e % 16];
        }
        if (++nflush % 8 == 0) {
#pragma unroll
          for (int e = 0; e < C::N; ++e) { acc3[e * NR + t] += acc2[e]; acc2[e] = 0.f; }
        }
      }
      tc::fence_before_sync();
    };
    unsigned epar[2] = {0u, 0u};
    bool pend[2] = {false, false}, dirty[2] = {false, false};
    auto wait_empty = [&](int b) {
      if (!pend[b]) return;
      if (!tc::mbar_wait(empty + b, epar[b], kQWaitNs)) bad = 1;
      epar[b] ^= 1u;
      pend[b] = false;
    };
    if (nchunk > 0) issue(0);
    cp_async_commit();
    if (nchunk > 1) issue(1);
    cp_async_commit();
    for (int ch = 0; ch < nchunk; ++ch) {
      cp_async_wait<1>();  // chunk ch has landed (this thread's copies)
      const int b = ch & 1, set = (ch >> 1) & 1;
      wait_empty(b);       // the products of chunk ch - 2 have read buffer b
      producers_sync();    // every copy of chunk ch; chunk ch - 1 fully formed
      if (*reinterpret_cast<volatile int *>(&bad)) break;
      if (ch + 2 < nchunk) issue(ch + 2);  // into the stage chunk ch - 1 came from
      cp_async_commit();
      if ((ch & 1) && ch >= 3 && dirty[set ^ 1]) {  // (restarted by chunk ch + 1)
        flush_set(set ^ 1);
        dirty[set ^ 1] = false;
      }
      const float *S = raw + (ch % kQS) * C::RAW;
      unsigned char *Ah = opbuf + (size_t)b * C::BUF * 4, *Al = Ah + C::OPA * 4;
      unsigned char *Bh = Al + C::OPA * 4, *Bl = Bh + C::OPB * 4;
      if (arole) {
#pragma unroll
        for (int p = 0; p < 8 / C::JA; ++p) {
          const int jg = ajg + C::JA * p, jj = 4 * jg;
          float4 x;
          if (avec) {
            x = *reinterpret_cast<const float4 *>(S + arow_s + jj);
          } else {
            const float4 sc = *reinterpret_cast<const float4 *>(S + arow_s + jj);
            const float4 a = *reinterpret_cast<const float4 *>(S + arow_c + jj);
            x = ashift ? make_float4(S[arow_c + jj - 1], a.x, a.y, a.z) : a;  // X_L: one cell back
            x.x *= sc.x;
            x.y *= sc.y;
            x.z *= sc.z;
            x.w *= sc.w;
          }
          float4 h, l;
          tc::split(x.x, h.x, l.x);
          tc::split(x.y, h.y, l.y);
          tc::split(x.z, h.z, l.z);
          tc::split(x.w, h.w, l.w);
          const uint32_t off = (uint32_t)((jg >> 1) * C::M * 32 + (jg & 1) * 128) + arow_o;
          *reinterpret_cast<float4 *>(Ah + off) = h;
          *reinterpret_cast<float4 *>(Al + off) = l;
        }
      } else if (brole) {
#pragma unroll
        for (int p = 0; p < 8 / C::JB; ++p) {
          const int jg = bjg + C::JB * p, jj = 4 * jg;
          const float4 x = *reinterpret_cast<const float4 *>(S + brow_c + jj);
          float4 h, l;
          tc::split(x.x, h.x, l.x);
          tc::split(x.y, h.y, l.y);
          tc::split(x.z, h.z, l.z);
          tc::split(x.w, h.w, l.w);
          const uint32_t off = (uint32_t)((jg >> 1) * C::N * 32 + (jg & 1) * 128) + brow_o;
          *reinterpret_cast<float4 *>(Bh + off) = h;
          *reinterpret_cast<float4 *>(Bl + off) = l;
        }
      }
      tc::fence_smem_to_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(full + b);
      pend[b] = true;
      dirty[set] = true;
    }
    // the last products: the older buffer's commit first, then the older
    // pair's set before the newer one
    if (nchunk > 0 && !*reinterpret_cast<volatile int *>(&bad)) {
      const int last = nchunk - 1;
      if (last >= 1) wait_empty((last - 1) & 1);
      wait_empty(last & 1);
      producers_sync();
      if (!*reinterpret_cast<volatile int *>(&bad)) {
        const int lset = (last >> 1) & 1;
        if (dirty[lset ^ 1]) flush_set(lset ^ 1);
        if (dirty[lset]) flush_set(lset);
      }
    }
    cp_async_wait<0>();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (bad && t == 0) set_status(I.status, kETimeout);
  if (w == 0) tc::dealloc(tmem, C::NCOL);
  // this CTA's partial (one per CTA, summed over the CTAs by k_reduce): D
  // row m (operand column) and column n (X column) give G_nj for
  // m = mat RB + j and the vector sums for m >= 6 RB, each from its owner
  double *out = I.partials + (size_t)blockIdx.x * proj_count(r);
  const int rr2 = r * r;
  if (reader) {
    const int m = 128 * (w >> 2) + 32 * (w & 3) + lane;
    if (m < 6 * RB) {
      const int mat = m / RB, j = m - mat * RB;
      const double sc = mat == 4 ? 4.0 * kPi : 1.0;
      if (j < r)
#pragma unroll
        for (int n = 0; n < C::N; ++n)
          if (n < r) out[mat * rr2 + n + r * j] = sc * ((double)acc2[n] + (double)acc3[n * NR + t]);
    } else if (m < 6 * RB + 5) {
      const int v = m - 6 * RB;
#pragma unroll
      for (int n = 0; n < C::N; ++n)
        if (n < r) out[6 * rr2 + v * r + n] = (double)acc2[n] + (double)acc3[n * NR + t];
    }
  }
}

// Sum of per-block partials: out[e] = scale * sum_b part[b*stride + e].
__global__ void __launch_bounds__(256) k_reduce(const ReduceJob *__restrict__ jobs) {
  pdl_wait();
  pdl_trigger();
  const ReduceJob J = jobs[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= J.count) return;
  J.out[e] = J.scale * sum_partials(J.part, J.nblocks, J.stride, e);
}

// ------------------------------------------------------------------
// step 9: T = T0 + dt sigma (phi - 4 pi B0) / D, phi = X (L w);
//         X0 <- X U (rotation to the SVD basis of S, columns signed)
// ------------------------------------------------------------------
template <typename real, int RB>
__global__ void __launch_bounds__(128) k_tupdate(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  if (rank_class(I.r) != RB) return;
  __shared__ real Us[RB * RB];
  __shared__ real vp[RB];
  const int r = I.r;
  const double *U = I.small + I.lay.U;
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int i = e % RB, j = e / RB;
    Us[e] = (i < r && j < r) ? real(U[i + r * j]) : real(0);
  }
  for (int e = threadIdx.x; e < RB; e += blockDim.x)
    vp[e] = e < r ? real(I.small[I.lay.vphi + e]) : real(0);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= I.N) return;
  const real *X = as_c<real>(I.X);
  real x[RB];
  real phi = real(0);
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    x[i] = i < r ? X[(size_t)I.N * i + c] : real(0);
    phi += x[i] * vp[i];
  }
  real *X0 = as<real>(I.X0);
  for (int j = 0; j < r; ++j) {
    real v = real(0);
#pragma unroll
    for (int i = 0; i < RB; ++i) v += x[i] * Us[j * RB + i];
    X0[(size_t)I.N * j + c] = v;
  }
  const double T0 = I.T[c];
  const double T = T0 + I.dt * sigma_at(I, c, T0) * ((double)phi - 4.0 * kPi * I.B0[c]) / I.D[c];
  I.T[c] = T;
  if (!(T > 0.0)) {
    atomicAdd(I.nonpos, 1);
    if (!I.allow_nonpos) set_status(I.status, kENonPos);
  }
}

// ------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------
// one launch per rank class in mask (bits: 8, 16, 32)
#define DLR_RB_DISPATCH(mask, MACRO)                   \
  do {                                                 \
    if ((mask) & 1) MACRO(8);                          \
    if (e == cudaSuccess && ((mask) & 2)) MACRO(16);   \
    if (e == cudaSuccess && ((mask) & 4)) MACRO(32);   \
  } while (0)

template <typename real>
cudaError_t launch_coeff_recon(const Inst *d, int n, int maxN, int rmask, int grp_mode, cudaStream_t st) {
  dim3 g((maxN + 255) / 256, n);
#define L_(RB) (e = launch_pdl(k_coeff_recon<real, RB>, g, dim3(256), 0, st, d, grp_mode))
  cudaError_t e = cudaSuccess;
  DLR_RB_DISPATCH(rmask, L_);
#undef L_
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ------------------------------------------------------------------
// Gram of an FP32 column-major m x r matrix (r <= 32, no weights), for the
// CholeskyQR passes of step 5 in mixed precision: G = sum over rows of
// a a^T, one FP64 partial per thread-block cluster (both triangles).  Rows stream through a
// ring of kGS shared-memory stages of kGR rows filled by cp.async (16-byte
// chunks when lda is a multiple of 4, else 4-byte ones; rows past the CTA's
// slice are zero-filled), so several rounds are in flight per CTA and two
// CTAs share an SM.  A stage holds column c at c kGR, its rows rotated by
// 4 (c / 4 mod 8) so that the 16-byte reads of the eight column quads of a
// tile row fall in distinct banks.  Products as in k_tsgram: 4 x 4 register
// tiles on and above the diagonal, FP32 over about 64 rows per thread, then
// FP64; the CTA's row groups, then the cluster's CTAs (through distributed
// shared memory, rank order) are summed in a fixed order.  The tiles are
// packed so that every lane of a warp owns one (a square grid of tiles
// left the warps below the diagonal two-thirds idle).
// ------------------------------------------------------------------
constexpr int kGR = 128, kGS = 4;
constexpr int gram32_smem_bytes() { return kGS * 32 * kGR * 4; }
// position of (column c, row q) of a stage
__device__ __forceinline__ int g32_at(int c, int q) { return c * kGR + ((q + 4 * ((c >> 2) & 7)) & (kGR - 1)); }

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kTB, 2) k_gram32(const GramJob *__restrict__ jobs) {
  pdl_wait();
  pdl_trigger();
  const GramJob J = jobs[blockIdx.y];
  // nblocks is a multiple of the cluster size and run_if is per job, so
  // whole clusters leave together
  if ((int)blockIdx.x >= J.nblocks || (J.run_if && *J.run_if == 0)) return;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char gsm[];
  float *ring = reinterpret_cast<float *>(gsm);
  const float *A = as_c<float>(J.A);
  const int r = J.r, t = threadIdx.x, lda = J.lda;
  // the 4 x 4 tiles on and above the diagonal, packed: tile u = bj (bj + 1)
  // / 2 + bi (bi <= bj); kTB / ntile groups of threads split the rows
  const int side = (r + 3) >> 2, ntile = side * (side + 1) / 2;
  const int ngroup = kTB / ntile;
  const int grp = t / ntile, tt = t - grp * ntile;
  int bj = 0;
  while ((bj + 1) * (bj + 2) / 2 <= tt) ++bj;
  const int ti = 4 * (tt - bj * (bj + 1) / 2), tj = 4 * bj;
  const bool own = grp < ngroup;
  // slices of a multiple of 4 rows: with lda a multiple of 4 every 16-byte
  // chunk of a stage starts 16-byte aligned
  const int per = ((J.m + J.nblocks - 1) / J.nblocks + 3) & ~3;
  const int row0 = min(J.m, (int)blockIdx.x * per), row1 = min(J.m, row0 + per);
  const int nround = (row1 - row0 + kGR - 1) / kGR;
  const bool vec = (lda & 3) == 0 && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  auto load = [&](int rd) {
    float *st = ring + (size_t)(rd % kGS) * 32 * kGR;
    const int base = row0 + rd * kGR;
    if (vec) {
      for (int c = t; c < r * (kGR / 4); c += kTB) {
        const int i = c / (kGR / 4), q = c - i * (kGR / 4);
        const int row = base + 4 * q;
        const int n_ok = max(0, min(4, row1 - row));  // rows of the chunk in the slice
        // a chunk past the slice reads nothing (zero-filled) from an aligned
        // address inside the matrix
        cp_async16(st + g32_at(i, 4 * q), A + (size_t)lda * i + (n_ok > 0 ? row : row0), 4 * n_ok);
      }
    } else {
      for (int c = t; c < r * kGR; c += kTB) {
        const int i = c / kGR, q = c - i * kGR;
        const int row = base + q;
        const bool ok = row < row1;
        cp_async4(st + g32_at(i, q), A + (size_t)lda * i + (ok ? row : row1 - 1), ok ? 4 : 0);
      }
    }
  };
  const int flush_every = max(1, 64 * ngroup / kGR);
  float s[16];
  double acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) { s[e] = 0.f; acc[e] = 0.0; }
#pragma unroll
  for (int p = 0; p < kGS - 1; ++p) {
    if (p < nround) load(p);
    cp_async_commit();
  }
  for (int rd = 0; rd < nround; ++rd) {
    cp_async_wait<kGS - 2>();
    __syncthreads();  // stage rd has landed; stage rd - 1 is no longer read
    if (rd + kGS - 1 < nround) load(rd + kGS - 1);
    cp_async_commit();
    const float *st = ring + (size_t)(rd % kGS) * 32 * kGR;
    if (own) {
      const int nq = (min(kGR, row1 - row0 - rd * kGR) + 3) >> 2;  // quads holding rows
      for (int q = grp; q < nq; q += ngroup) {
        Quad<float> a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // columns past r (r not a multiple of 4) read a valid column;
          // those tile entries are never written out
          a[k] = *reinterpret_cast<const Quad<float> *>(st + g32_at(min(ti + k, r - 1), 4 * q));
          b[k] = *reinterpret_cast<const Quad<float> *>(st + g32_at(min(tj + k, r - 1), 4 * q));
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < 4; ++m) s[kk * 4 + k] += a[kk].v[m] * b[k].v[m];
      }
      if ((rd + 1) % flush_every == 0 || rd + 1 == nround) {
#pragma unroll
        for (int e = 0; e < 16; ++e) { acc[e] += (double)s[e]; s[e] = 0.f; }
      }
    }
  }
  cp_async_wait<0>();
  // groups -> CTA partial in a fixed order, the lower triangle mirrored
  __syncthreads();
  double *buf = reinterpret_cast<double *>(gsm);
  double *part_s = buf + kTB * 16;
  if (grp < ngroup) {
#pragma unroll
    for (int e = 0; e < 16; ++e) buf[t * 16 + e] = acc[e];
  }
  __syncthreads();
  for (int e = t; e < r * r; e += kTB) {
    int i = e % r, j = e / r;
    if (i > j) { const int x = i; i = j; j = x; }
    const int tl = (j >> 2) * ((j >> 2) + 1) / 2 + (i >> 2), comp = (i & 3) * 4 + (j & 3);
    double v = 0.0;
    for (int g = 0; g < ngroup; ++g) v += buf[(g * ntile + tl) * 16 + comp];
    part_s[e] = v;
  }
  cluster.sync();
  // this CTA's share of the cluster sum, CTA partials added in rank order
  const int rank = (int)cluster.block_rank();
  const int rr2 = r * r, share = (rr2 + kCl - 1) / kCl;
  double *out = J.out + (size_t)(blockIdx.x / kCl) * rr2;
  for (int e = rank * share + t; e < min(rr2, (rank + 1) * share); e += kTB) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < kCl; ++q) v += cluster.map_shared_rank(part_s, q)[e];
    out[e] = v;
  }
  cluster.sync();  // peers' shared memory stays valid until every read is done
}

cudaError_t launch_gram32(const GramJob *d_jobs, int n, int maxblocks, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gram32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         gram32_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_gram32, dim3(maxblocks, n), dim3(kTB), gram32_smem_bytes(), st, d_jobs);
}

// CTAs of k_gram32 that can be resident at once (whole clusters), or 0.
int gram32_cta_cap() {
  if (cudaFuncSetAttribute(k_gram32, cudaFuncAttributeMaxDynamicSharedMemorySize, gram32_smem_bytes()) !=
      cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCl);
  cfg.blockDim = dim3(kTB);
  cfg.dynamicSmemBytes = gram32_smem_bytes();
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int c = 0;
  if (cudaOccupancyMaxActiveClusters(&c, k_gram32, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return c * kCl;
}

// layout: the (common) layout of the batch's matrices
template <typename real>
cudaError_t launch_tsgram(const GramJob *d_jobs, int n, int maxblocks, int layout, cudaStream_t st) {
  if (layout == 0) return launch_pdl(k_tsgram<real, 0>, dim3(maxblocks, n), dim3(kTB), 0, st, d_jobs);
  return launch_pdl(k_tsgram<real, 1>, dim3(maxblocks, n), dim3(kTB), 0, st, d_jobs);
}

template <typename real>
cudaError_t launch_fill(const FillJob *d_jobs, int n, int maxm, cudaStream_t st) {
  return launch_pdl(k_fill<real>, dim3((maxm + 255) / 256, n), dim3(256), 0, st, d_jobs);
}

template <typename rin, typename rout>
cudaError_t launch_apply(const ApplyJob *d_jobs, int n, int maxm, int rmask, cudaStream_t st) {
  dim3 g((maxm + 127) / 128, n);
#define L_(RB) (e = launch_pdl(k_apply<rin, rout, RB>, g, dim3(128), 0, st, d_jobs))
  cudaError_t e = cudaSuccess;
  DLR_RB_DISPATCH(rmask, L_);
#undef L_
  return e != cudaSuccess ? e : cudaGetLastError();
}

// FP64: k_project; mixed precision: k_project_tc5, one launch per rank
// class in rmask
template <typename real>
cudaError_t launch_project(const Inst *d, int n, int maxblocks, int rmax, int rmask, cudaStream_t st) {
  if (sizeof(real) == 8)
    return launch_pdl(k_project<double>, dim3(maxblocks, n), dim3(kTB), proj_smem_bytes(rmax, 8), st, d);
  const dim3 g(maxblocks, n);
#define L_(RB) (e = launch_pdl(k_project_tc5<RB>, g, dim3(kQT), Q5<RB>::SMEM, st, d))
  cudaError_t e = cudaSuccess;
  DLR_RB_DISPATCH(rmask, L_);
#undef L_
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t prepare_dense(int rmax);

// Clusters of the reduction kernels that can be resident at once (the CTA
// count of a reduction is kept to that many clusters, so it runs in one
// wave); 0 if it cannot be determined.
int reduce_cluster_cap() {
  auto cap = [](const void *fn, size_t smem, int threads = kTB) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  };
  int c = cap((const void *)k_tsgram<float, 0>, 0);
  c = std::min(c, cap((const void *)k_tsgram<double, 0>, 0));
  c = std::min(c, cap((const void *)k_tsgram<double, 1>, 0));
  if (prepare_dense(kMaxRank) == cudaSuccess)
    c = std::min(c, cap((const void *)k_project<double>, proj_smem_bytes(kMaxRank, 8)));
  return c;
}

// Kernel attributes, set before any launch is captured into a graph.
cudaError_t prepare_dense(int rmax) {
  cudaError_t e = cudaFuncSetAttribute(k_project_tc5<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Q5<8>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_project_tc5<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q5<16>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_project_tc5<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, Q5<32>::SMEM);

  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_project<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              proj_smem_bytes(rmax, 8));
}

cudaError_t launch_reduce(const ReduceJob *d_jobs, int n, int maxcount, cudaStream_t st) {
  return launch_pdl(k_reduce, dim3((maxcount + 255) / 256, n), dim3(256), 0, st, d_jobs);
}

template <typename real>
cudaError_t launch_tupdate(const Inst *d, int n, int maxN, int rmask, cudaStream_t st) {
  dim3 g((maxN + 127) / 128, n);
#define L_(RB) (e = launch_pdl(k_tupdate<real, RB>, g, dim3(128), 0, st, d))
  cudaError_t e = cudaSuccess;
  DLR_RB_DISPATCH(rmask, L_);
#undef L_
  return e != cudaSuccess ? e : cudaGetLastError();
}

template cudaError_t launch_coeff_recon<float>(const Inst *, int, int, int, int, cudaStream_t);
template cudaError_t launch_coeff_recon<double>(const Inst *, int, int, int, int, cudaStream_t);
template cudaError_t launch_tsgram<float>(const GramJob *, int, int, int, cudaStream_t);
template cudaError_t launch_tsgram<double>(const GramJob *, int, int, int, cudaStream_t);
template cudaError_t launch_fill<float>(const FillJob *, int, int, cudaStream_t);
template cudaError_t launch_fill<double>(const FillJob *, int, int, cudaStream_t);
template cudaError_t launch_apply<float, float>(const ApplyJob *, int, int, int, cudaStream_t);
template cudaError_t launch_apply<double, double>(const ApplyJob *, int, int, int, cudaStream_t);
template cudaError_t launch_project<float>(const Inst *, int, int, int, int, cudaStream_t);
template cudaError_t launch_project<double>(const Inst *, int, int, int, int, cudaStream_t);
template cudaError_t launch_tupdate<float>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_tupdate<double>(const Inst *, int, int, int, cudaStream_t);

}  // namespace dlr
