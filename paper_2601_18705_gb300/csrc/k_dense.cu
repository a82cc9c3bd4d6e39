// k_dense.cu -- per-cell and tall-skinny kernels of the SN-like DLR step
// (Algorithm 1 of Haut et al.):
//   k_coeff_recon  step 1 (Newton-linearised sigma_s, q of Section 2.2) and
//                  step 3 (psi0_j = sum_k X0_k L0_k(Om^(j))), fused with the
//                  fixed source q + psi0_j/(c dt) of the collocation system
//                  and the starting scalar flux gamma^T Psi0
//   k_tsgram       G = sum_c wt_c a_c a_c^T for a tall-skinny matrix (step 5
//                  CholeskyQR Grams of Psi and step 8 Grams of L)
//   k_apply        out = diag(s_out) (diag(s_in) A) T for a small dense T
//   k_project      step 6 P = <X, X0> and the step 7 Galerkin operators:
//                  Gram, x/y neighbour Grams, <sigma_t X, X>, <sigma_s X, X>,
//                  <q, X> and the four edge sums
//   k_tupdate      step 9 temperature update (Eq. temperature update, Newton
//                  form) with phi = X (L w), fused with the rotation X0 <- X U
// Mixed precision: products and sums over a chunk of kChunk cells in FP32,
// chunk sums accumulated in FP64.
#include "dlr_internal.cuh"

namespace dlr {

constexpr int kChunk = 256;   // cells per FP32 partial sum
constexpr int kTB = 256;      // threads per block of the reduction kernels

// ------------------------------------------------------------------
// step 1 + step 3
// ------------------------------------------------------------------
template <typename real, int RB>
__global__ void __launch_bounds__(256) k_coeff_recon(const Inst *__restrict__ insts) {
  const Inst &I = insts[blockIdx.y];
  __shared__ real C0s[RB * RB];
  __shared__ real gam[RB];
  const int r = I.r;
  const double *C0 = I.small + I.lay.C0;
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int k = e % RB, j = e / RB;  // C0s[j*RB + k] = C0[k, j]
    C0s[e] = (k < r && j < r) ? real(C0[k + r * j]) : real(0);
  }
  for (int e = threadIdx.x; e < RB; e += blockDim.x)
    gam[e] = e < r ? real(I.small[I.lay.gamma + e]) : real(0);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= I.N) return;
  // Section 2.2 (Newton linearisation, B = a c T^4 / 4pi)
  const double T0 = I.T[c], sig = I.sigma[c], rho = I.rho_cv[c];
  const double B = I.a_rad * I.c * T0 * T0 * T0 * T0 / (4.0 * kPi);
  const double dB = I.a_rad * I.c * T0 * T0 * T0 / kPi;
  const double g = 4.0 * kPi * I.dt * sig * dB;
  const double D = rho + g;
  const double ss = sig * g / D;
  const double q = sig * B - sig * dB * (4.0 * kPi * I.dt * sig * B) / D;
  I.B0[c] = B;
  I.D[c] = D;
  as<real>(I.sig_t)[c] = real(sig + I.inv_cdt);
  const real ss4 = real(ss / (4.0 * kPi));
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
    s0[(size_t)I.N * j + c] = qr + icdt * p;
    phi += gam[j] * p;
  }
  as<real>(I.phi0)[c] = phi;
  as<real>(I.sphi)[c] = ss4 * phi;
}

// ------------------------------------------------------------------
// tall-skinny Gram with 2x2 register tiles per thread (r <= 32)
// ------------------------------------------------------------------
// A is m x r; layout 0: column-major A[row + lda*i]; layout 1: rows of r
// contiguous A[i + r*row].  wt: per-row weight or nullptr.  Each block
// writes its partial r x r sum (FP64, column-major) to out + blockIdx.x*r*r.

template <typename real>
__global__ void __launch_bounds__(kTB) k_tsgram(const GramJob *__restrict__ jobs) {
  const GramJob J = jobs[blockIdx.y];
  if ((int)blockIdx.x >= J.nblocks || (J.run_if && *J.run_if == 0)) return;
  __shared__ real tile[kChunk / 8][33];  // 32 rows x r columns
  __shared__ real tileb[kChunk / 8][33];
  __shared__ real wts[kChunk / 8];
  const int r = J.r;
  const int t = threadIdx.x;
  // 2x2 tiles of G; for small r, G groups of threads split the rows
  const int side = (r + 1) / 2, ntile = side * side;
  const int ngroup = max(1, (int)blockDim.x / ntile);
  const int grp = t / ntile, tt = t % ntile;
  const int ti = (tt % side) * 2, tj = (tt / side) * 2;
  const bool own = grp < ngroup;
  double acc[4] = {0, 0, 0, 0};
  const real *A = as_c<real>(J.A);
  __shared__ double gsum[256 * 4];
  const int chunk = J.chunk;
  const int nchunks = (J.m + chunk - 1) / chunk;
  for (int ch = blockIdx.x; ch < nchunks; ch += J.nblocks) {
    real s[4] = {0, 0, 0, 0};
    for (int sub = 0; sub < chunk; sub += 32) {
      const int row0 = ch * chunk + sub;
      __syncthreads();
      for (int e = t; e < 32 * r; e += blockDim.x) {
        int rr, i;
        if (J.layout == 0) { rr = e & 31; i = e >> 5; }
        else { i = e % r; rr = e / r; }
        const int row = row0 + rr;
        real v = real(0);
        if (row < J.m) v = J.layout == 0 ? A[(size_t)J.lda * i + row] : A[(size_t)r * row + i];
        tile[rr][i] = v;
      }
      if (J.B) {
        const real *Bm = as_c<real>(J.B);
        for (int e = t; e < 32 * r; e += blockDim.x) {
          const int rr = e & 31, i = e >> 5, row = row0 + rr;
          tileb[rr][i] = row < J.m ? Bm[(size_t)J.ldb * i + row] : real(0);
        }
      }
      if (t < 32) {
        const int row = row0 + t;
        double wv = (row < J.m) ? (J.wt ? J.wt[row] : 1.0) : 0.0;
        if (J.sqrt_wt) wv = sqrt(wv);
        wts[t] = real(wv);
      }
      __syncthreads();
      if (own) {
        for (int rr = grp; rr < 32; rr += ngroup) {
          const real w = wts[rr];
          const real a0 = tile[rr][ti] * w, a1 = tile[rr][ti + 1] * w;
          const real b0 = J.B ? tileb[rr][tj] : tile[rr][tj];
          const real b1 = J.B ? tileb[rr][tj + 1] : tile[rr][tj + 1];
          s[0] += a0 * b0; s[1] += a1 * b0; s[2] += a0 * b1; s[3] += a1 * b1;
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += (double)s[e];
  }
  // combine the groups in a fixed order
  __syncthreads();
  if (own && grp > 0)
    for (int e = 0; e < 4; ++e) gsum[((grp - 1) * ntile + tt) * 4 + e] = acc[e];
  __syncthreads();
  if (own && grp == 0) {
    for (int g = 1; g < ngroup; ++g)
      for (int e = 0; e < 4; ++e) acc[e] += gsum[((g - 1) * ntile + tt) * 4 + e];
    double *o = J.out + (size_t)blockIdx.x * r * r;
    if (ti < r && tj < r) o[ti + r * tj] = acc[0];
    if (ti + 1 < r && tj < r) o[ti + 1 + r * tj] = acc[1];
    if (ti < r && tj + 1 < r) o[ti + r * (tj + 1)] = acc[2];
    if (ti + 1 < r && tj + 1 < r) o[ti + 1 + r * (tj + 1)] = acc[3];
  }
}

// ------------------------------------------------------------------
// orthonormal completion: dependent columns replaced by pseudo-random ones
// ------------------------------------------------------------------
__device__ __forceinline__ double hash_uniform(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <typename real>
__global__ void __launch_bounds__(256) k_fill(const FillJob *__restrict__ jobs) {
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
  const ApplyJob J = jobs[blockIdx.y];
  if (J.run_if && *J.run_if == 0) return;
  __shared__ rout Ts[RB * RB];
  const int r = J.r;
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int i = e % RB, j = e / RB;
    Ts[e] = (i < r && j < r) ? rout(J.T[i + r * j]) : rout(0);
  }
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
  for (int j = 0; j < r; ++j) {
    rout v = rout(0);
#pragma unroll
    for (int i = 0; i < RB; ++i) v += a[i] * Ts[j * RB + i];
    O[(size_t)J.ldo * j + row] = so * v;
  }
}

// ------------------------------------------------------------------
// step 6 / step 7 projections.  Per block partial (FP64) layout, r x r
// column-major each: G, Nx, Ny, Mt, Ms, P, then vec[5r]: qh, bL, bR, bB, bT.
//   G_ij  = sum_c X_ci X_cj            Mt_ij = sum_c sig_t X_ci X_cj
//   Ms_ij = sum_c sigma_s X_ci X_cj    P_ij  = sum_c X_ci X0_cj
//   Nx_ij = sum_{ix>=1} X_ci X_{c-1,j} Ny_ij = sum_{iy>=1} X_ci X_{c-nx,j}
// (all without the h^2 factor, applied in the reduction)
// ------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kTB) k_project(const Inst *__restrict__ insts) {
  const Inst &I = insts[blockIdx.y];
  if ((int)blockIdx.x >= I.partial_blocks) return;
  constexpr int CR = 32;  // cells per staging round
  __shared__ real xs[CR + 1][33];   // cells c0-1 .. c0+31
  __shared__ real xb[CR][33];       // cells c0-nx .. c0-nx+31
  __shared__ real x0s[CR][33];
  __shared__ real sts[CR], sss[CR], qs[CR];
  __shared__ int ixs[CR], iys[CR];
  const int r = I.r, N = I.N, nx = I.nx;
  const int t = threadIdx.x;
  const int side = (r + 1) / 2, ntile = side * side;
  const int ngroup = ntile <= 64 ? (int)blockDim.x / ntile : 1;  // groups split the cells
  const int grp = t / ntile, tt = t % ntile;
  const int ti = (tt % side) * 2, tj = (tt / side) * 2;
  const bool own = grp < ngroup;
  const real *X = as_c<real>(I.X), *X0 = as_c<real>(I.X0);
  const real *sig_t = as_c<real>(I.sig_t), *ss4 = as_c<real>(I.ss4), *qv = as_c<real>(I.q);
  double acc[6][4];
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[a][e] = 0.0;
  double vacc[5] = {0, 0, 0, 0, 0};  // thread t < r: qh, bL, bR, bB, bT for index t
  const real four_pi = real(4.0 * kPi);
  const int nchunks = (N + kChunk - 1) / kChunk;
  for (int ch = blockIdx.x; ch < nchunks; ch += I.partial_blocks) {
    real s[6][4];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) s[a][e] = real(0);
    real vs[5] = {0, 0, 0, 0, 0};
    for (int sub = 0; sub < kChunk; sub += CR) {
      const int c0 = ch * kChunk + sub;
      __syncthreads();
      for (int e = t; e < (CR + 1) * r; e += blockDim.x) {
        const int cc = e % (CR + 1), i = e / (CR + 1);
        const int c = c0 - 1 + cc;
        xs[cc][i] = (c >= 0 && c < N) ? X[(size_t)N * i + c] : real(0);
      }
      for (int e = t; e < CR * r; e += blockDim.x) {
        const int cc = e & (CR - 1), i = e / CR;
        const int c = c0 + cc, cb = c - nx;
        xb[cc][i] = (cb >= 0 && c < N) ? X[(size_t)N * i + cb] : real(0);
        x0s[cc][i] = (c < N) ? X0[(size_t)N * i + c] : real(0);
      }
      if (t < CR) {
        const int c = c0 + t;
        const bool in = c < N;
        sts[t] = in ? sig_t[c] : real(0);
        sss[t] = in ? ss4[c] * four_pi : real(0);
        qs[t] = in ? qv[c] : real(0);
        ixs[t] = in ? c % nx : -1;
        iys[t] = in ? c / nx : -1;
      }
      __syncthreads();
      if (own) {
        for (int cc = grp; cc < CR; cc += ngroup) {
          const int ix = ixs[cc], iy = iys[cc];
          if (ix < 0) break;
          const real a0 = xs[cc + 1][ti], a1 = xs[cc + 1][ti + 1];
          const real b0 = xs[cc + 1][tj], b1 = xs[cc + 1][tj + 1];
          const real st = sts[cc], sg = sss[cc];
          const real p00 = a0 * b0, p10 = a1 * b0, p01 = a0 * b1, p11 = a1 * b1;
          s[0][0] += p00; s[0][1] += p10; s[0][2] += p01; s[0][3] += p11;
          s[3][0] += st * p00; s[3][1] += st * p10; s[3][2] += st * p01; s[3][3] += st * p11;
          s[4][0] += sg * p00; s[4][1] += sg * p10; s[4][2] += sg * p01; s[4][3] += sg * p11;
          if (ix >= 1) {
            const real l0 = xs[cc][tj], l1 = xs[cc][tj + 1];
            s[1][0] += a0 * l0; s[1][1] += a1 * l0; s[1][2] += a0 * l1; s[1][3] += a1 * l1;
          }
          if (iy >= 1) {
            const real d0 = xb[cc][tj], d1 = xb[cc][tj + 1];
            s[2][0] += a0 * d0; s[2][1] += a1 * d0; s[2][2] += a0 * d1; s[2][3] += a1 * d1;
          }
          const real o0 = x0s[cc][tj], o1 = x0s[cc][tj + 1];
          s[5][0] += a0 * o0; s[5][1] += a1 * o0; s[5][2] += a0 * o1; s[5][3] += a1 * o1;
        }
      }
      if (t < r) {
        for (int cc = 0; cc < CR; ++cc) {
          const int ix = ixs[cc], iy = iys[cc];
          if (ix < 0) break;
          const real x = xs[cc + 1][t];
          vs[0] += qs[cc] * x;
          if (ix == 0) vs[1] += x;
          if (ix == nx - 1) vs[2] += x;
          if (iy == 0) vs[3] += x;
          if (iy == I.ny - 1) vs[4] += x;
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][e] += (double)s[a][e];
#pragma unroll
    for (int e = 0; e < 5; ++e) vacc[e] += (double)vs[e];
  }
  double *o = I.partials + (size_t)blockIdx.x * proj_count(r);
  // combine the groups in a fixed order (stage through the partial slot)
  __shared__ double gsum[6 * 4 * 64];
  for (int g = 1; g < ngroup; ++g) {
    __syncthreads();
    if (own && grp == g && tt < 64)
      for (int a = 0; a < 6; ++a)
        for (int e = 0; e < 4; ++e) gsum[(a * 4 + e) * 64 + tt] = acc[a][e];
    __syncthreads();
    if (own && grp == 0 && tt < 64)
      for (int a = 0; a < 6; ++a)
        for (int e = 0; e < 4; ++e) acc[a][e] += gsum[(a * 4 + e) * 64 + tt];
  }
  if (own && grp == 0) {
    for (int a = 0; a < 6; ++a) {
      double *m = o + (size_t)a * r * r;
      if (ti < r && tj < r) m[ti + r * tj] = acc[a][0];
      if (ti + 1 < r && tj < r) m[ti + 1 + r * tj] = acc[a][1];
      if (ti < r && tj + 1 < r) m[ti + r * (tj + 1)] = acc[a][2];
      if (ti + 1 < r && tj + 1 < r) m[ti + 1 + r * (tj + 1)] = acc[a][3];
    }
  }
  if (t < r) {
    double *v = o + 6 * r * r;
    for (int e = 0; e < 5; ++e) v[e * r + t] = vacc[e];
  }
}

// Sum of per-block partials: out[e] = scale * sum_b part[b*stride + e].
__global__ void __launch_bounds__(256) k_reduce(const ReduceJob *__restrict__ jobs) {
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
  const Inst &I = insts[blockIdx.y];
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
  const double T = T0 + I.dt * I.sigma[c] * ((double)phi - 4.0 * kPi * I.B0[c]) / I.D[c];
  I.T[c] = T;
  if (!(T > 0.0)) {
    atomicAdd(I.nonpos, 1);
    if (!I.allow_nonpos) set_status(I.status, kENonPos);
  }
}

// ------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------
#define DLR_RB_DISPATCH(r, MACRO) \
  ((r) <= 8 ? MACRO(8) : (r) <= 16 ? MACRO(16) : MACRO(32))

template <typename real>
cudaError_t launch_coeff_recon(const Inst *d, int n, int maxN, int r, cudaStream_t st) {
  dim3 g((maxN + 255) / 256, n);
#define L_(RB) (k_coeff_recon<real, RB><<<g, 256, 0, st>>>(d), 0)
  DLR_RB_DISPATCH(r, L_);
#undef L_
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_tsgram(const GramJob *d_jobs, int n, int maxblocks, cudaStream_t st) {
  k_tsgram<real><<<dim3(maxblocks, n), kTB, 0, st>>>(d_jobs);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fill(const FillJob *d_jobs, int n, int maxm, cudaStream_t st) {
  k_fill<real><<<dim3((maxm + 255) / 256, n), 256, 0, st>>>(d_jobs);
  return cudaGetLastError();
}

template <typename rin, typename rout>
cudaError_t launch_apply(const ApplyJob *d_jobs, int n, int maxm, int r, cudaStream_t st) {
  dim3 g((maxm + 127) / 128, n);
#define L_(RB) (k_apply<rin, rout, RB><<<g, 128, 0, st>>>(d_jobs), 0)
  DLR_RB_DISPATCH(r, L_);
#undef L_
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_project(const Inst *d, int n, int maxblocks, cudaStream_t st) {
  k_project<real><<<dim3(maxblocks, n), kTB, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceJob *d_jobs, int n, int maxcount, cudaStream_t st) {
  k_reduce<<<dim3((maxcount + 255) / 256, n), 256, 0, st>>>(d_jobs);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_tupdate(const Inst *d, int n, int maxN, int r, cudaStream_t st) {
  dim3 g((maxN + 127) / 128, n);
#define L_(RB) (k_tupdate<real, RB><<<g, 128, 0, st>>>(d), 0)
  DLR_RB_DISPATCH(r, L_);
#undef L_
  return cudaGetLastError();
}

template cudaError_t launch_coeff_recon<float>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_coeff_recon<double>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_tsgram<float>(const GramJob *, int, int, cudaStream_t);
template cudaError_t launch_tsgram<double>(const GramJob *, int, int, cudaStream_t);
template cudaError_t launch_fill<float>(const FillJob *, int, int, cudaStream_t);
template cudaError_t launch_fill<double>(const FillJob *, int, int, cudaStream_t);
template cudaError_t launch_apply<float, float>(const ApplyJob *, int, int, int, cudaStream_t);
template cudaError_t launch_apply<double, double>(const ApplyJob *, int, int, int, cudaStream_t);
template cudaError_t launch_project<float>(const Inst *, int, int, cudaStream_t);
template cudaError_t launch_project<double>(const Inst *, int, int, cudaStream_t);
template cudaError_t launch_tupdate<float>(const Inst *, int, int, int, cudaStream_t);
template cudaError_t launch_tupdate<double>(const Inst *, int, int, int, cudaStream_t);

}  // namespace dlr
