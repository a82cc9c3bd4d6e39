// k_sn.cu -- the full-rank SN step that Algorithm 1 approximates (the
// comparison method of Section 5): the same DG0 upwind sweeps and source
// iteration as Algorithm 1 step 4, but over every angle of the quadrature
// with phi = sum_k w_k psi_k, followed by the temperature update of
// Section 2.2.  The sweeps and the iteration are k_si itself (r = NOm
// swept angles, idx the identity, gamma = w); these kernels supply its
// inputs and consume its scalar flux:
//   k_sn_init     psi = B(T0) at every cell and angle (isotropic equilibrium)
//   k_sn_prep     coefficients of Section 2.2, fixed sources
//                 q + psi^n_k / (c dt) for all k, starting scalar flux
//                 phi^n = sum_k w_k psi^n_k
//   k_sn_tupdate  T = T0 + dt sigma (phi - 4 pi B0) / D with the scalar flux
//                 of the last source iteration
#include <algorithm>

#include "dlr_internal.cuh"

namespace dlr {

template <typename real>
__global__ void __launch_bounds__(256) k_sn_init(real *__restrict__ psi, const double *__restrict__ T,
                                                 int N, int K, double a_rad, double c_light) {
  const size_t total = (size_t)N * K;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double T0 = T[e % N];
    psi[e] = real(a_rad * c_light * T0 * T0 * T0 * T0 / (4.0 * kPi));
  }
}

template <typename real>
__global__ void __launch_bounds__(256) k_sn_prep(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= I.N) return;
  const CellCoef cf = cell_coefficients(I, c);
  I.B0[c] = cf.B;
  I.D[c] = cf.D;
  as<real>(I.sig_t)[c] = real(cf.sig + I.inv_cdt);
  const real ss4 = real(cf.ss / (4.0 * kPi));
  as<real>(I.ss4)[c] = ss4;
  as<real>(I.q)[c] = real(cf.q);
  const real *psi = as_c<real>(I.Psi);
  real *s0 = as<real>(I.s0);
  const real qr = real(cf.q), icdt = real(I.inv_cdt);
  real phi = real(0);
  const int ix = c % I.nx, iy = c / I.nx, L = I.nx + I.ny;
  for (int k = 0; k < I.K; ++k) {
    const real p = psi[(size_t)I.N * k + c];
    real v = fmadd(icdt, p, qr);
    if (I.refl_base) {
      // reflective edges: keep the boundary cell's own source and add the
      // inflow of the first iteration, from psi^n of the mirror directions
      const ReflGeom<real> G(I, k);
      real *base = as<real>(I.refl_base) + (size_t)k * L;
      const real f = v;
      if (G.rx && ix == G.bx) {
        base[iy] = f;
        v = fmadd(G.ax, psi[(size_t)I.N * mirror_angle(k, I.n_azim, 0) + c], v);
      }
      if (G.ry && iy == G.by) {
        base[I.ny + ix] = f;
        v = fmadd(G.ay, psi[(size_t)I.N * mirror_angle(k, I.n_azim, 1) + c], v);
      }
    }
    s0[(size_t)I.N * k + c] = v;
    phi = fmadd(real(I.w[k]), p, phi);
  }
  as<real>(I.phi0)[c] = phi;
  as<real>(I.sphi)[c] = ss4 * phi;
}

template <typename real>
__global__ void __launch_bounds__(256) k_sn_tupdate(const Inst *__restrict__ insts) {
  pdl_wait();
  pdl_trigger();
  const Inst &I = insts[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= I.N) return;
  // iteration it writes its new scalar flux to phi1 (it even) or phi0 (odd)
  const int last = *I.iters - 1;
  const real *phi = as_c<real>((last & 1) ? I.phi0 : I.phi1);
  const double T0 = I.T[c];
  const double T = T0 + I.dt * sigma_at(I, c, T0) * ((double)phi[c] - 4.0 * kPi * I.B0[c]) / I.D[c];
  I.T[c] = T;
  if (!(T > 0.0)) {
    atomicAdd(I.nonpos, 1);
    if (!I.allow_nonpos) set_status(I.status, kENonPos);
  }
}

template <typename real>
cudaError_t launch_sn_init(void *psi, const double *T, int N, int K, double a_rad, double c_light,
                           cudaStream_t st) {
  const size_t total = (size_t)N * K;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
  k_sn_init<real><<<blocks, 256, 0, st>>>(static_cast<real *>(psi), T, N, K, a_rad, c_light);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_sn_prep(const Inst *d, int n, int maxN, cudaStream_t st) {
  return launch_pdl(k_sn_prep<real>, dim3((maxN + 255) / 256, n), dim3(256), 0, st, d);
}

template <typename real>
cudaError_t launch_sn_tupdate(const Inst *d, int n, int maxN, cudaStream_t st) {
  return launch_pdl(k_sn_tupdate<real>, dim3((maxN + 255) / 256, n), dim3(256), 0, st, d);
}

template cudaError_t launch_sn_init<float>(void *, const double *, int, int, double, double, cudaStream_t);
template cudaError_t launch_sn_init<double>(void *, const double *, int, int, double, double, cudaStream_t);
template cudaError_t launch_sn_prep<float>(const Inst *, int, int, cudaStream_t);
template cudaError_t launch_sn_prep<double>(const Inst *, int, int, cudaStream_t);
template cudaError_t launch_sn_tupdate<float>(const Inst *, int, int, cudaStream_t);
template cudaError_t launch_sn_tupdate<double>(const Inst *, int, int, cudaStream_t);

}  // namespace dlr
