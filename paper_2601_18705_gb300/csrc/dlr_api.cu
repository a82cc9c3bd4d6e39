// dlr_api.cu -- the C ABI of include/dlr.h: handle lifetime, the initial
// factors, batch plans (device-side work descriptors for all instances of a
// batch) and the launch sequence of one SN-like DLR step (Algorithm 1 of
// Haut et al.):
//   graph "pre":  select angles (step 2), coefficients + psi0 (steps 1, 3),
//                 source-iteration control reset
//   direct:       cooperative source-iteration kernel (step 4)
//   graph "post": CholeskyQR of Psi (step 5), projections (steps 6, 7),
//                 L-step (step 7), CholeskyQR + SVD of L (step 8),
//                 temperature update and factor rotation (step 9)
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/dlr.h"
#include "dlr_internal.cuh"

namespace dlr {
// launchers defined in the kernel translation units
template <typename real> cudaError_t launch_si(const Inst *, const SiCtl &, int, cudaStream_t);
template <typename real> int si_max_grid(int, int, int, int, int);
int si_sweep_warps(bool mixed);
int si_sweep_lag(bool mixed);
cudaError_t launch_grp_prep(const Inst *, int, const SiCtl &, GrpSi *, cudaStream_t);
cudaError_t launch_grp_iteration(const Inst *, int, const SiCtl &, GrpSi *, int grid, int stages,
                                 cudaGraphConditionalHandle loop, cudaStream_t);
cudaError_t launch_grp_final(const Inst *, const SiCtl &, GrpSi *, int grid, int stages, cudaStream_t);
int si_grp_stages(int nx_max, int bands_max, int n_inst);
int si_grp_max_grid(int nx_max, int bands_max, int n_inst, int stages);
int si_grp_warps();
int si_grp_lag();
template <typename real> size_t si_smem_bytes(int, int, int, int, int);
template <typename real> cudaError_t launch_sn_init(void *, const double *, int, int, double, double, cudaStream_t);
template <typename real> cudaError_t launch_sn_prep(const Inst *, int, int, cudaStream_t);
template <typename real> cudaError_t launch_sn_tupdate(const Inst *, int, int, cudaStream_t);
template <typename real>
cudaError_t launch_sweep_dirs(int, int, double, double, int, const double *, const double *,
                              const real *, const real *, real *, int *, cudaStream_t);
template <typename real> cudaError_t launch_coeff_recon(const Inst *, int, int, int, int, cudaStream_t);
cudaError_t launch_gram32(const GramJob *, int, int maxblocks, cudaStream_t);
int gram32_cta_cap();
template <typename real> cudaError_t launch_tsgram(const GramJob *, int, int, int, cudaStream_t);
template <typename real> cudaError_t launch_fill(const FillJob *, int, int, cudaStream_t);
template <typename rin, typename rout>
cudaError_t launch_apply(const ApplyJob *, int, int, int, cudaStream_t);
template <typename real> cudaError_t launch_project(const Inst *, int, int, int, int, cudaStream_t);
cudaError_t prepare_dense(int);
cudaError_t prepare_lside(int, int);
int lside_max_k();
cudaError_t launch_lside(const Inst *, int, int, int, cudaStream_t);
int reduce_cluster_cap();
cudaError_t launch_reduce(const ReduceJob *, int, int, cudaStream_t);
template <typename real> cudaError_t launch_tupdate(const Inst *, int, int, int, cudaStream_t);
cudaError_t launch_select(const Inst *, int, int, cudaStream_t);
cudaError_t launch_chol(const CholJob *, const Inst *, int, cudaStream_t);
cudaError_t launch_proj_post(const Inst *, int, cudaStream_t);
size_t lstep_angle_smem(int);
cudaError_t launch_lstep(const Inst *, int, int, int, int, int, cudaStream_t);
cudaError_t launch_svd(const Inst *, int, int, cudaStream_t);
cudaError_t launch_sign(const Inst *, int, int, cudaStream_t);
cudaError_t launch_si_prep(const Inst *, int, SiCtl, cudaStream_t);
cudaError_t prepare_small(int, int, int);
cudaError_t launch_aug_pad(const Inst *, int, cudaStream_t);
cudaError_t launch_aug_trunc(const Inst *, int, cudaStream_t);
template <typename real> cudaError_t launch_refl_pre(const Inst *, int, int, int, cudaStream_t);
template <typename real> cudaError_t launch_refl_kap(const Inst *, int, int, int, cudaStream_t);
template <typename real> cudaError_t launch_refl_lstep(const Inst *, int, cudaStream_t);
template <typename real> cudaError_t launch_q1_coeff(const Inst *, int, int, bool, cudaStream_t);
template <typename real> size_t q1_si_smem(int, int, int, int);
template <typename real> int q1_si_max_grid(int, int, int, int);
template <typename real> cudaError_t launch_q1_si(const Inst *, const SiCtl &, int, cudaStream_t);
template <typename real> cudaError_t launch_q1_transport(const Inst *, int, int, int, cudaStream_t);
template <typename real> cudaError_t launch_q1_vec(const Inst *, int, int, cudaStream_t);
template <typename real> cudaError_t launch_q1_tupdate(const Inst *, int, int, bool, cudaStream_t);
cudaError_t launch_q1_rescale(void *, bool, size_t, int, int, cudaStream_t);
}  // namespace dlr

using namespace dlr;

// FP32 <-> FP64 column copies of X
__global__ void k_widen(const float *a, double *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
__global__ void k_narrow(const double *a, float *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// psi = X S W^T of a DLR state (Section 4: the low-rank form of the angular
// flux), FP64, column-major rows x K: CTA (bx, k) forms l = S W_k^T (r
// values) and then rows 128 bx .. of column k; X in the working precision
// (Q1 coefficients stored scaled are returned plain)
template <typename real>
__global__ void __launch_bounds__(128) k_form_psi(const real *__restrict__ X, size_t rows, int r,
                                                  const double *__restrict__ S, const double *__restrict__ W,
                                                  int K, int q1, double *__restrict__ out) {
  __shared__ double l[32];
  const int k = blockIdx.y;
  if (threadIdx.x < r) {
    double v = 0.0;
    for (int j = 0; j < r; ++j) v += S[threadIdx.x + r * j] * W[k + (size_t)K * j];
    l[threadIdx.x] = v;
  }
  __syncthreads();
  const size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (row >= rows) return;
  double v = 0.0;
  for (int i = 0; i < r; ++i) v += (double)X[row + rows * i] * l[i];
  out[row + rows * k] = q1 ? v * q1_unscale((int)(row & 3)) : v;
}


// ------------------------------------------------------------------
// errors
// ------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

namespace dlr {
// lets other translation units report through dlr_last_error()
int record_error(int code, const char *msg) {
  g_err = msg ? msg : "";
  return code;
}
}  // namespace dlr

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(DLR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                  __FILE__, __LINE__);                                                \
  } while (0)

static const char *status_name(int s) {
  switch (s) {
    case DLR_ENOTCONV: return "source iteration did not converge within si_max_iter";
    case DLR_ESINGULAR: return "singular collocation or L-step matrix";
    case DLR_ETIMEOUT: return "a bounded device-side wait ran out";
    case DLR_ENONPOS: return "temperature became non-positive";
    default: return "device error";
  }
}

// ------------------------------------------------------------------
// handle and batch plan
// ------------------------------------------------------------------
struct Batch;

struct dlr_handle {
  dlr_problem prob{};
  int N = 0, K = 0, r = 0;
  bool mixed = false;
  size_t rs = 8;  // sizeof(real)
  cudaStream_t st = nullptr;
  bool own_stream = false;
  dlr_runtime rt{};
  std::vector<void *> allocs;
  Inst inst{};
  unsigned version = 0;  // bumped whenever inst changes on the host
  std::vector<double> ox, oy, oz, w;
  int pb = 1;    // partial blocks of the cell reductions
  int pbg = 1;   // CTAs of the FP32 Grams of step 5
  int pbl = 1;   // partial blocks of the angle reductions
  int lb = 1;    // blocks of the per-angle L-step
  // device counters: [0] total SI iterations
  long long *d_iters_total = nullptr;
  long long *d_dsa_iters_total = nullptr;  // CG iterations of the DSA solves
  int *h_status = nullptr;  // pinned mirror of the device status
  int64_t steps = 0;
  bool timing = false;
  double ms_si = 0, ms_step = 0;
  int64_t si_launches = 0;
  int64_t kernel_launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::array<cudaEvent_t, 4>> ev_pending;
  Batch *own_batch = nullptr;
  bool canonical = true;  // S0 diagonal (SVD basis) since the last step
  bool sn = false;        // full-rank SN instance (r = K swept angles)
  bool grp_loop = false;  // the last step took the grouped source iteration
  bool aug = false;       // augmented step: steps 5-10 on inst2 at rank 2r
  Inst inst2{};
};

struct Batch {
  std::vector<dlr_handle *> hs;
  std::vector<unsigned> versions;  // handle versions of the uploaded copies
  int n = 0;
  bool mixed = false;
  cudaStream_t st = nullptr;
  Inst *d_insts = nullptr;   // contiguous copies of the instances
  void *d_mem = nullptr;     // jobs, units, control
  int maxN = 0, maxK = 0, rmax = 0, pbmax = 1, pblmax = 1, lbmax = 1, pbgmax = 1;
  int rmask_pre = 0, rmask = 0;  // rank classes of steps 1-4 and of steps 5-10
  int nx_max = 0, bands_max = 0, si_grid = 0;
  SiCtl ctl{};
  SiUnit *d_units = nullptr;  // capacity units_cap
  int spare_row = 0;          // an edge row no unit writes (dlr_debug_lose_edge)
  int units_cap = 0;
  double split = 0;           // splitting threshold of the unit plan (<= 0: no split)
  bool sn = false;            // a batch of full-rank SN instances
  bool aug = false;           // a batch of augmented instances (steps 5-10 on d_insts2)
  Inst *d_insts2 = nullptr;   // the instances of steps 5-10 (rank 2r when augmented)
  int sel_slice_max = 1;      // most angles one CTA of the selection cluster owns
  bool lside_fused = false;   // step 8 by the one-cluster kernel (pivoted-QR choice, K <= lside_max_k())
  bool refl = false;          // some DLR instance has reflective edges (k_reflect.cu)
  bool q1 = false;            // a batch of bilinear-element instances (k_q1.cu)
  int maxRows = 0;            // most rows of X (4 N with Q1 elements)
  GramJob *g_q1t = nullptr;   // Q1: X^T (T X) per axis direction (4 n), then M_t, M_s, P (3 n)
  ReduceJob *r_q1 = nullptr;  // Q1: the seven reductions (7 n)
  int maxL = 0;               // most boundary entries nx + ny
  bool grp_ok = false;        // every instance can take the grouped sweep (k_sweepg.cu)
  bool grp = false;           // ... and the batch takes it
  int grid_angle = 0, grid_grp = 0;  // CTAs of the per-angle and the grouped sweep
  int grp_stages = 0;         // shared-memory stages per warp of the grouped sweep
  GrpSi *gs = nullptr;        // its loop state (device)
  cudaGraphExec_t si = nullptr;  // its source iteration: a while node and the last sweep
  GramJob *g_psi1, *g_psire, *g_x, *g_x3, *g_l1, *g_lf, *g_w, *g_w3, *g_cross;
  FillJob *f_psi, *f_l;
  ApplyJob *a_psi, *a_x2, *a_x3, *a_l1, *a_w2, *a_w3, *a_wv, *a_cw, *a_cx;
  int svd_mode = 0;  // 0: S kept general (pivoted-QR selection), 1: SVD every step (DEIM, r = NOm)
  CholJob *c_p1, *c_p1b, *c_p2, *c_p3, *c_l1, *c_l1b, *c_l2, *c_l3;
  ReduceJob *r_proj;
  cudaGraphExec_t pre = nullptr, post = nullptr;
  int kernels_per_step = 0;  // kernel launches of one step (graphs + direct)
  int kcount = 0;            // counter used while capturing
};

static void *dev_alloc(dlr_handle *h, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void *p = nullptr;
  if (h->rt.alloc) {
    p = h->rt.alloc(bytes, h->rt.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) h->allocs.push_back(p);
  return p;
}

static void dev_free_all(dlr_handle *h) {
  for (void *p : h->allocs) {
    if (h->rt.free) h->rt.free(p, h->rt.ctx);
    else if (!h->rt.alloc) cudaFree(p);
  }
  h->allocs.clear();
}

// ------------------------------------------------------------------
// quadrature and initial factors (host, FP64)
// ------------------------------------------------------------------
static void gl_nodes(int n, std::vector<double> &x, std::vector<double> &wt) {
  // roots of P_n by Newton from cos(pi (i + 3/4) / (n + 1/2)); weights
  // 2 / ((1 - x^2) P_n'(x)^2); ascending
  x.assign(n, 0.0);
  wt.assign(n, 0.0);
  auto pn = [n](double z, double &d) {
    double p0 = 1.0, p1 = z;
    if (n == 0) { d = 0.0; return 1.0; }
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    d = n * (z * p1 - p0) / (z * z - 1.0);
    return p1;
  };
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), d = 0.0;
    for (int it = 0; it < 200; ++it) {
      double p = pn(z, d);
      double dz = p / d;
      z -= dz;
      if (std::fabs(dz) < 1e-15) {
        p = pn(z, d);
        z -= p / d;
        break;
      }
    }
    pn(z, d);
    x[n - 1 - i] = z;
    wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * d * d);
  }
}

static void build_quadrature(dlr_handle *h) {
  const int np = h->prob.n_polar, na = h->prob.n_azim;
  std::vector<double> mu, wp;
  gl_nodes(np, mu, wp);
  h->ox.resize(h->K);
  h->oy.resize(h->K);
  h->oz.resize(h->K);
  h->w.resize(h->K);
  for (int p = 0; p < np; ++p) {
    const double s = std::sqrt(1.0 - mu[p] * mu[p]);
    for (int a = 0; a < na; ++a) {
      const double ph = (a + 0.5) * 2.0 * kPi / na;
      const int k = p * na + a;
      h->ox[k] = s * std::cos(ph);
      h->oy[k] = s * std::sin(ph);
      h->oz[k] = mu[p];
      h->w[k] = wp[p] * 2.0 * kPi / na;
    }
  }
}

// W0: monomials Om_x^a Om_y^b by total degree (a descending), then the same
// times Om_z, orthonormalised in sum_k w_k (two modified Gram-Schmidt
// passes, candidates with < 1e-8 surviving are skipped).  Returns false if
// fewer than r independent candidates exist.
static bool build_W0(const dlr_handle *h, std::vector<double> &W) {
  const int K = h->K, r = h->r;
  W.assign((size_t)K * r, 0.0);
  std::vector<double> v(K);
  int cnt = 0;
  for (int e = 0; e <= 1 && cnt < r; ++e)
    for (int d = 0; d <= 12 && cnt < r; ++d)
      for (int a = d; a >= 0 && cnt < r; --a) {
        const int b = d - a;
        double n0 = 0.0;
        for (int k = 0; k < K; ++k) {
          v[k] = std::pow(h->ox[k], a) * std::pow(h->oy[k], b) * (e ? h->oz[k] : 1.0);
          n0 += h->w[k] * v[k] * v[k];
        }
        n0 = std::sqrt(n0);
        if (n0 == 0.0) continue;
        for (int pass = 0; pass < 2; ++pass)
          for (int l = 0; l < cnt; ++l) {
            double dd = 0.0;
            for (int k = 0; k < K; ++k) dd += h->w[k] * W[k + (size_t)K * l] * v[k];
            for (int k = 0; k < K; ++k) v[k] -= dd * W[k + (size_t)K * l];
          }
        double n1 = 0.0;
        for (int k = 0; k < K; ++k) n1 += h->w[k] * v[k] * v[k];
        n1 = std::sqrt(n1);
        if (n1 > 1e-8 * n0) {
          for (int k = 0; k < K; ++k) W[k + (size_t)K * cnt] = v[k] / n1;
          ++cnt;
        }
      }
  return cnt == r;
}

// X0: first column f / |f| with f = B(T0) (the only column that carries
// psi0, since S0 = diag(s0, 0, ...)); the others are the DCT modes
// cos(pi k x^) cos(pi l y^), (k, l) != (0, 0) in (k + l, k) order, reflected
// by the Householder map that swaps the constant mode and f / |f|, which
// keeps them orthonormal and orthogonal to f.  All in the h^2 inner product.
// r columns (at most N).
static bool build_X0(const dlr_handle *h, const double *T0, int r, std::vector<double> &X, double &fn) {
  const int nx = h->prob.nx, ny = h->prob.ny, N = h->N;
  const double hx = h->prob.lx / nx, hy = h->prob.ly / ny, h2 = hx * hy;
  X.assign((size_t)N * r, 0.0);
  std::vector<double> f(N), u(N, 1.0 / std::sqrt(h->prob.lx * h->prob.ly)), v(N);
  fn = 0.0;
  for (int c = 0; c < N; ++c) {
    f[c] = h->prob.a_rad * h->prob.c * std::pow(T0[c], 4) / (4.0 * kPi);
    fn += h2 * f[c] * f[c];
  }
  fn = std::sqrt(fn);
  std::vector<double> fh(N);
  for (int c = 0; c < N; ++c) fh[c] = fn > 0 ? f[c] / fn : u[c];
  double vv = 0.0;
  for (int c = 0; c < N; ++c) {
    v[c] = u[c] - fh[c];
    vv += h2 * v[c] * v[c];
  }
  auto reflect = [&](std::vector<double> &m) {
    if (vv <= 0.0) return;
    double d = 0.0;
    for (int c = 0; c < N; ++c) d += h2 * v[c] * m[c];
    for (int c = 0; c < N; ++c) m[c] -= 2.0 * d / vv * v[c];
  };
  for (int c = 0; c < N; ++c) X[c] = fh[c];
  int cnt = 1;
  std::vector<double> m(N), cx, cy;
  for (int d = 1; d <= nx + ny - 2 && cnt < r; ++d)
    for (int k = 0; k <= d && cnt < r; ++k) {
      const int l = d - k;
      if (k >= nx || l >= ny) continue;
      const double ck = std::sqrt((k == 0 ? 1.0 : 2.0) / h->prob.lx);
      const double cl = std::sqrt((l == 0 ? 1.0 : 2.0) / h->prob.ly);
      cx.resize(nx);
      cy.resize(ny);
      for (int ix = 0; ix < nx; ++ix) cx[ix] = ck * std::cos(kPi * k * (ix + 0.5) / nx);
      for (int iy = 0; iy < ny; ++iy) cy[iy] = cl * std::cos(kPi * l * (iy + 0.5) / ny);
      for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) m[iy * nx + ix] = cx[ix] * cy[iy];
      reflect(m);
      for (int c = 0; c < N; ++c) X[c + (size_t)N * cnt] = m[c];
      ++cnt;
    }
  return cnt == r;
}

// ------------------------------------------------------------------
// footprint
// ------------------------------------------------------------------
struct Sizes {
  int N, K, r, pb, pbl, lb;
  int pbg;  // CTAs (and partials) of the FP32 Grams of step 5 (k_gram32; mixed precision)
  size_t rs;
  size_t partial_doubles;
  size_t total;
};

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// CTAs a reduction may use: whole clusters, all resident at once
static int reduce_cta_cap() {
  static int cap = 0;
  if (!cap) {
    const int c = reduce_cluster_cap();
    cap = c > 0 ? c * kCl : 15 * kCl;
  }
  return cap;
}

// The grouped sweep (k_sweepg.cu) serves mixed-precision DLR steps on DG0
// cells without DSA, reflective edges or the augmented step, unless
// sweep_mode asks for the per-angle kernel.
static bool grp_eligible(const dlr_problem *p) {
  return p->precision == DLR_MIXED && p->method == DLR_METHOD_DLR && !p->dsa && !p->augment &&
         !(p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3]) && p->sweep_mode != 1 &&
         p->element == 0;
}

static Sizes sizes_of(const dlr_problem *p, int sms) {
  Sizes s;
  s.N = p->nx * p->ny;
  s.K = p->n_polar * p->n_azim;
  s.r = p->rank;
  s.rs = p->precision == DLR_MIXED ? 4 : 8;
  if (p->method == DLR_METHOD_SN) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    s.r = s.K;
    s.pb = s.pbl = s.lb = kCl;
    s.pbg = 1;
    s.partial_doubles = 0;
    s.total = 5 * al((size_t)s.N * 8) + 6 * al((size_t)s.N * s.rs) + 2 * al((size_t)s.N * s.K * s.rs) +
              3 * al((size_t)s.K * 8) + al((size_t)s.K * 4) + al(64) * 4 + al(sizeof(Inst));
    if (p->dsa) s.total += kDsaArrays * al((size_t)s.N * s.rs) + al(64);
    if (p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3])
      s.total += al((size_t)s.K * (p->nx + p->ny) * s.rs);  // boundary sources of reflective edges
    if (p->element == 1)  // Q1: psi, s0 and phi with 4 coefficients per cell
      s.total += 2 * al((size_t)3 * s.N * s.K * s.rs) + 2 * al((size_t)3 * s.N * s.rs);
    return s;
  }
  // CTAs of the cell and angle reductions: whole clusters of kCl CTAs,
  // about 512 cells or 16 angles per CTA
  const int cap = std::min(reduce_cta_cap(), 2 * sms / kCl * kCl);
  auto clusters = [&](int x) { return std::min(cap, (x + kCl - 1) / kCl * kCl); };
  s.pb = clusters(std::max(1, (s.N + 511) / 512));
  // mixed-precision DG0 steps use pb only for the projections of steps 6
  // and 7 (k_project_tc5): one CTA per SM at most, no clusters, one partial
  // per CTA, about 2048 cells per CTA
  const bool proj_tc = p->precision == DLR_MIXED && p->element == 0;
  if (proj_tc) s.pb = std::min(sms, std::max(1, (s.N + 2047) / 2048));
  s.pbl = clusters(std::max(1, (s.K + 15) / 16));
  s.lb = std::min(2 * sms / kCl * kCl, (std::max(1, (s.K + 3) / 4) + kCl - 1) / kCl * kCl);  // 4 warps, one angle each
  const size_t r1 = s.r;
  const size_t r = p->augment ? 2 * r1 : r1;    // rank of steps 5-10
  // the FP32 Grams (k_gram32): whole clusters, all resident at once (two
  // CTAs per SM), at least 2048 rows per CTA
  {
    static int gcap = 0;
    if (!gcap) gcap = std::max(kCl, gram32_cta_cap());
    s.pbg = std::min(gcap, std::max(kCl, (s.N / 2048) / kCl * kCl));
  }
  s.partial_doubles = std::max({(size_t)(proj_tc ? s.pb : s.pb / kCl) * proj_count((int)r),
                                (size_t)(s.pb / kCl) * r * r,
                                (size_t)(s.pbl / kCl) * r * r, (size_t)(s.lb / kCl) * (r * r + r),
                                (size_t)(s.pbg / kCl) * r * r,
                                p->element == 1 ? (size_t)7 * (s.pb / kCl) * r * r : (size_t)0,
                                p->element == 1 ? (size_t)s.pb * r : (size_t)0});
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t t = 0;
  t += 5 * al((size_t)s.N * 8);                 // sigma, rho_cv, T, B0, D
  t += 6 * al((size_t)s.N * s.rs);              // sig_t, ss4, q, phi0, phi1, sphi
  t += 3 * al((size_t)s.N * r * s.rs);          // X0, X, Psi (with X0 beside it when augmented)
  t += al((size_t)s.N * r1 * s.rs);             // s0
  t += 3 * al((size_t)s.K * 8);                 // ox, oy, w
  t += 3 * al((size_t)s.K * r * 8);             // W0, L, Lf
  t += al(r * r * 8) + al(r * 4);               // S0, idx
  t += al((size_t)small_layout((int)r).total * 8); // small
  if (p->augment) t += al(r1 * r1 * 8) + al((size_t)small_layout((int)r1).total * 8);  // rank-r S0, small
  t += al((size_t)s.K * r * r * 8) + al((size_t)s.K * r * 4);  // lu, piv
  t += al(s.partial_doubles * 8);
  t += al(64) * 4 + al(sizeof(Inst));           // status, iters, conv, totals, inst
  if (p->dsa) t += kDsaArrays * al((size_t)s.N * s.rs) + al(64);  // DSA coefficients, CG vectors
  if (p->element == 1)  // Q1: X0, X, Psi, s0, phi with 4 rows per cell, Gram weights, T X
    t += 3 * al((size_t)3 * s.N * r * s.rs) + al((size_t)3 * s.N * r1 * s.rs) + 2 * al((size_t)3 * s.N * s.rs) +
         2 * al((size_t)4 * s.N * 8) + al((size_t)4 * s.N * r * s.rs);
  if (p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3]) {
    const size_t LB = (size_t)p->nx + p->ny;
    t += al(r1 * LB * s.rs) + al(2 * LB * r1 * 8) + al((size_t)s.K * LB * 8) + 2 * al((size_t)s.K * r1 * 8) +
         al(64);  // boundary sources, What^-1 Psi, boundary values, y_k, u_k, passes
  }
  if (grp_eligible(p)) {  // skewed inputs and partials of the grouped sweep
    const size_t L = grp_lay(p->nx, p->ny) * 4;
    const size_t ng = grp_count((int)r1);
    t += al(ng * (kGA + 1) * L) + al(8 * L) + al(ng * L) + al(4 * L) + al(ng * kGrpRec * 4);
  }
  s.total = t;
  return s;
}

size_t dlr_footprint_bytes(const dlr_problem *p) {
  if (!p || p->nx < 1 || p->ny < 1 || p->rank < 1 || p->n_polar < 1 || p->n_azim < 1) return 0;
  return sizes_of(p, num_sms()).total;
}

const char *dlr_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------
// create / destroy
// ------------------------------------------------------------------
static int validate(const dlr_problem *p) {
  if (!p) return fail(DLR_EINVAL, "problem is NULL");
  if (p->nx < 1 || p->ny < 1) return fail(DLR_EINVAL, "nx, ny must be >= 1");
  if (!(p->lx > 0) || !(p->ly > 0)) return fail(DLR_EINVAL, "lx, ly must be > 0");
  if (p->n_polar < 1 || p->n_azim < 1) return fail(DLR_EINVAL, "n_polar, n_azim must be >= 1");
  const long long N = (long long)p->nx * p->ny, K = (long long)p->n_polar * p->n_azim;
  if (N > (1ll << 30) || K > 8192) return fail(DLR_EINVAL, "mesh or quadrature too large");
  if (p->method != DLR_METHOD_DLR && p->method != DLR_METHOD_SN) return fail(DLR_EINVAL, "bad method");
  if (!std::isfinite(p->sigma_texp) || !std::isfinite(p->cv_texp) || !std::isfinite(p->T_ref))
    return fail(DLR_EINVAL, "material exponents and T_ref must be finite");
  const bool sn = p->method == DLR_METHOD_SN;
  if (sn && N * K > (1ll << 34)) return fail(DLR_EINVAL, "nx*ny*NOm too large for a full-rank state");
  const long long rows = p->element == 1 ? 4 * N : N;  // rows of X (Q1: 4 coefficients per cell)
  if (!sn && (p->rank < 1 || p->rank > kMaxRank || p->rank > rows || p->rank > K))
    return fail(DLR_EINVAL, "rank must satisfy 1 <= r <= min(%d, rows of X, NOm)", kMaxRank);
  if (!(p->dt > 0) || !(p->c > 0) || !(p->a_rad >= 0)) return fail(DLR_EINVAL, "dt, c must be > 0, a_rad >= 0");
  if (p->precision != DLR_FP64 && p->precision != DLR_MIXED) return fail(DLR_EINVAL, "bad precision");
  if (p->selection != DLR_SEL_QDEIM && p->selection != DLR_SEL_DEIM) return fail(DLR_EINVAL, "bad selection");
  if (p->augment != 0 && p->augment != 1) return fail(DLR_EINVAL, "augment must be 0 or 1");
  if (p->augment == 1) {
    if (sn) return fail(DLR_EINVAL, "the augmented step is a DLR mode");
    if (2 * p->rank > kMaxRank || 2 * p->rank > N || 2 * p->rank > K)
      return fail(DLR_EINVAL, "augmented step: 2r must be <= min(%d, nx*ny, NOm)", kMaxRank);
    if (K > 1024 || p->selection != DLR_SEL_QDEIM)
      return fail(DLR_EINVAL, "augmented step: needs NOm <= 1024 and the pivoted-QR angle choice");
  }
  if (p->dsa != 0 && p->dsa != 1) return fail(DLR_EINVAL, "dsa must be 0 or 1");
  for (int e = 0; e < 4; ++e)
    if (p->reflect[e] != 0 && p->reflect[e] != 1) return fail(DLR_EINVAL, "reflect[%d] must be 0 or 1", e);
  if (p->sweep_mode < 0 || p->sweep_mode > 2) return fail(DLR_EINVAL, "sweep_mode must be 0, 1 or 2");
  if (p->element != 0 && p->element != 1) return fail(DLR_EINVAL, "element must be 0 or 1");
  if (p->element == 1) {
    if (p->dsa || p->augment || p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3])
      return fail(DLR_EINVAL, "bilinear elements: no DSA, augmented step or reflective edges");
    if (!sn && p->selection != DLR_SEL_QDEIM)
      return fail(DLR_EINVAL, "bilinear elements need the pivoted-QR angle choice");
  }
  if (p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3]) {
    if (p->augment) return fail(DLR_EINVAL, "reflective edges are not built for the augmented step");
    if ((p->reflect[0] || p->reflect[1]) && p->n_azim % 2)
      return fail(DLR_EINVAL, "a reflective left or right edge needs an even n_azim");
  }
  if (!std::isfinite(p->dsa_tol) || p->dsa_tol >= 1.0) return fail(DLR_EINVAL, "dsa_tol must be finite and < 1");
  if (!p->sigma || !p->rho_cv || !p->T0) return fail(DLR_EINVAL, "sigma, rho_cv, T0 must be given");
  for (long long c = 0; c < N; ++c) {
    if (!(p->sigma[c] >= 0) || !std::isfinite(p->sigma[c])) return fail(DLR_EINVAL, "sigma[%lld] invalid", c);
    if (!(p->rho_cv[c] > 0) || !std::isfinite(p->rho_cv[c])) return fail(DLR_EINVAL, "rho_cv[%lld] invalid", c);
    if (!(p->T0[c] > 0) || !std::isfinite(p->T0[c])) return fail(DLR_EINVAL, "T0[%lld] invalid", c);
  }
  // shared memory of the sweep for this mesh
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int gam = sn ? (int)K : kMaxRank;
  const size_t need = p->precision == DLR_MIXED ? si_smem_bytes<float>(p->nx, (p->ny + 31) / 32, 256, gam, p->dsa)
                                                : si_smem_bytes<double>(p->nx, (p->ny + 31) / 32, 256, gam, p->dsa);
  if (optin > 0 && need > (size_t)optin) return fail(DLR_EINVAL, "nx = %d too large for the sweep's shared memory", p->nx);
  const size_t need_q1 = p->precision == DLR_MIXED ? q1_si_smem<float>(p->nx, (p->ny + 31) / 32, 256, gam)
                                                   : q1_si_smem<double>(p->nx, (p->ny + 31) / 32, 256, gam);
  if (p->element == 1 && optin > 0 && need_q1 > (size_t)optin)
    return fail(DLR_EINVAL, "nx = %d too large for the bilinear sweep's shared memory", p->nx);
  return DLR_OK;
}

static double planck(double a, double c, double T) { return a * c * T * T * T * T / (4.0 * kPi); }

static void destroy_batch(Batch *b);
static void purge_batches(dlr_handle *h);

static void fill_common(dlr_handle *h, const dlr_problem *problem) {
  Inst &I = h->inst;
  I.nx = problem->nx;
  I.ny = problem->ny;
  I.N = h->N;
  I.r = h->r;
  I.K = h->K;
  I.precision = problem->precision;
  I.selection = problem->selection;
  I.fixed_iters = problem->si_fixed_iters > 0 ? problem->si_fixed_iters : 0;
  I.max_iter = problem->si_max_iter > 0 ? problem->si_max_iter : 1000;
  I.hx = problem->lx / problem->nx;
  I.hy = problem->ly / problem->ny;
  I.h2 = I.hx * I.hy;
  I.dt = problem->dt;
  I.c = problem->c;
  I.a_rad = problem->a_rad;
  I.inv_cdt = 1.0 / (problem->c * problem->dt);
  I.si_tol = problem->si_tol > 0 ? problem->si_tol : (h->mixed ? 1e-6 : 1e-13);
  for (int e = 0; e < 4; ++e)
    I.psi_edge[e] = problem->T_edge[e] >= 0 ? planck(problem->a_rad, problem->c, problem->T_edge[e]) : 0.0;
  I.method = problem->method;
  I.gamma_ext = nullptr;
  I.sig_texp = problem->sigma_texp;
  I.cv_texp = problem->cv_texp;
  I.T_ref = problem->T_ref > 0 ? problem->T_ref : 1.0;
  // DSA (Section 4.5): penalty kappa = (1/8 pi) sum_k w_k |Om_k . n| per face
  // orientation; the stencil coefficients are scaled by 1/h^2
  I.dsa = problem->dsa;
  I.dsa_tol = problem->dsa_tol > 0 ? problem->dsa_tol : 0.1;
  I.dsa_max_iter = problem->dsa_max_iter > 0 ? problem->dsa_max_iter : 3;
  double kx = 0, ky = 0;
  for (int k = 0; k < h->K; ++k) {
    kx += h->w[k] * std::fabs(h->ox[k]);
    ky += h->w[k] * std::fabs(h->oy[k]);
  }
  kx /= 8.0 * kPi;
  ky /= 8.0 * kPi;
  I.dsa_cx = 1.0 / (12.0 * I.hx * I.hx);
  I.dsa_cy = 1.0 / (12.0 * I.hy * I.hy);
  I.dsa_kx = kx / I.hx;
  I.dsa_ky = ky / I.hy;
  I.dsa_ist = I.dsa_dg = I.dsa_dinv = I.dsa_x = I.dsa_r = I.dsa_z = I.dsa_p0 = I.dsa_p1 = I.dsa_q = nullptr;
  I.dsa_iters_total = nullptr;
  for (int e = 0; e < 4; ++e) I.reflect[e] = problem->reflect[e];
  I.n_azim = problem->n_azim;
  {
    // polar pairs for step 7: an even n_polar whose mirrored polar levels
    // give bitwise equal Om_x, Om_y (the Gauss nodes are symmetric)
    const int np = problem->n_polar, na = problem->n_azim;
    bool pairs = np % 2 == 0 && np >= 2;
    for (int p = 0; pairs && p < np / 2; ++p)
      for (int a = 0; a < na; ++a) {
        const int k = p * na + a, kp = (np - 1 - p) * na + a;
        if (h->ox[k] != h->ox[kp] || h->oy[k] != h->oy[kp]) pairs = false;
      }
    I.polar_pairs = pairs ? 1 : 0;
  }
  I.refl_base = nullptr;
  I.refl_kap = I.refl_data = I.refl_y = I.refl_u = nullptr;
  I.refl_passes = nullptr;
  I.q1 = problem->element == 1 ? 1 : 0;
  I.q1_wt = I.q1_ws = nullptr;
  I.q1_v = nullptr;
  I.grp = 0;
  I.grp_ng = 0;
  I.grp_tab = nullptr;
  I.sgk = I.spk = I.part = I.qsum = nullptr;
}

// Device arrays of the DSA solve (N each, working precision): 1/sigma_t,
// the diagonal and its inverse, x, r, z, two search directions, q.
template <typename Alloc>
static void alloc_dsa(dlr_handle *h, Alloc &A) {
  Inst &I = h->inst;
  if (!I.dsa) return;
  const size_t b = (size_t)h->N * h->rs;
  void **v[kDsaArrays] = {&I.dsa_ist, &I.dsa_dg, &I.dsa_dinv, &I.dsa_x, &I.dsa_r,
                          &I.dsa_z, &I.dsa_p0, &I.dsa_p1, &I.dsa_q};
  for (int k = 0; k < kDsaArrays; ++k) *v[k] = A(b);
  I.dsa_iters_total = (unsigned long long *)A(64);
  h->d_dsa_iters_total = (long long *)I.dsa_iters_total;
}

// Full-rank SN handle: the per-cell state of Algorithm 1's sweeps, psi and
// its fixed sources at every angle (N x K each), the quadrature, and the
// identity as the "selected" angles; psi starts at B(T0).
static int create_sn(dlr_handle *h, const dlr_problem *problem, dlr_handle **out) {
  h->sn = true;
  h->r = h->K;
  fill_common(h, problem);
  const int N = h->N, K = h->K;
  const size_t rs = h->rs;
  Inst &I = h->inst;
  I.lay = SmallLayout{};
  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = dev_alloc(h, bytes);
    ok = ok && p;
    return p;
  };
  double *sigma = (double *)A((size_t)N * 8);
  double *rho = (double *)A((size_t)N * 8);
  I.T = (double *)A((size_t)N * 8);
  I.B0 = (double *)A((size_t)N * 8);
  I.D = (double *)A((size_t)N * 8);
  I.sigma = sigma;
  I.rho_cv = rho;
  I.sig_t = A((size_t)N * rs);
  I.ss4 = A((size_t)N * rs);
  I.q = A((size_t)N * rs);
  const size_t rowsN = I.q1 ? (size_t)4 * N : (size_t)N;  // Q1: 4 coefficients per cell
  I.phi0 = A(rowsN * rs);
  I.phi1 = A(rowsN * rs);
  I.sphi = A((size_t)N * rs);
  I.Psi = A(rowsN * K * rs);
  I.s0 = A(rowsN * K * rs);
  if (I.reflect[0] || I.reflect[1] || I.reflect[2] || I.reflect[3])
    I.refl_base = A((size_t)K * (problem->nx + problem->ny) * rs);
  double *dox = (double *)A((size_t)K * 8), *doy = (double *)A((size_t)K * 8), *dw = (double *)A((size_t)K * 8);
  I.ox = dox;
  I.oy = doy;
  I.w = dw;
  I.gamma_ext = dw;
  I.idx = (int *)A((size_t)K * 4);
  I.status = (int *)A(64);
  I.nonpos = (int *)A(64);
  I.allow_nonpos = problem->allow_nonpositive ? 1 : 0;
  I.iters = (int *)A(64);
  I.conv = (unsigned long long *)A(64);
  h->d_iters_total = (long long *)A(64);
  I.iters_total = (unsigned long long *)h->d_iters_total;
  alloc_dsa(h, A);
  if (!ok) {
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return fail(DLR_ENOMEM, "device allocation failed");
  }
  if (cudaMallocHost(&h->h_status, sizeof(int)) != cudaSuccess) {
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return fail(DLR_ENOMEM, "pinned allocation failed");
  }
  *h->h_status = 0;
  std::vector<int> ident(K);
  for (int k = 0; k < K; ++k) ident[k] = k;
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st);
  };
  cudaError_t e = cudaSuccess;
  auto chain = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chain(up(sigma, problem->sigma, (size_t)N * 8));
  chain(up(rho, problem->rho_cv, (size_t)N * 8));
  chain(up(I.T, problem->T0, (size_t)N * 8));
  chain(up(dox, h->ox.data(), (size_t)K * 8));
  chain(up(doy, h->oy.data(), (size_t)K * 8));
  chain(up(dw, h->w.data(), (size_t)K * 8));
  chain(up(I.idx, ident.data(), (size_t)K * 4));
  chain(cudaMemsetAsync(I.status, 0, 64, h->st));
  chain(cudaMemsetAsync(I.nonpos, 0, 64, h->st));
  chain(cudaMemsetAsync(I.iters, 0, 64, h->st));
  chain(cudaMemsetAsync(h->d_iters_total, 0, 64, h->st));
  if (h->d_dsa_iters_total) chain(cudaMemsetAsync(h->d_dsa_iters_total, 0, 64, h->st));
  std::vector<double> psi_q1;
  if (I.q1) {
    // psi0 = B(T0) isotropic: each cell's constant coefficient, slopes zero
    psi_q1.assign(rowsN * K, 0.0);
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < N; ++c)
        psi_q1[(size_t)4 * c + rowsN * k] = planck(problem->a_rad, problem->c, problem->T0[c]);
    if (h->mixed) {
      std::vector<float> pf(psi_q1.begin(), psi_q1.end());
      chain(up(I.Psi, pf.data(), pf.size() * 4));
      chain(cudaStreamSynchronize(h->st));
    } else {
      chain(up(I.Psi, psi_q1.data(), psi_q1.size() * 8));
    }
  } else if (e == cudaSuccess) {
    e = h->mixed ? launch_sn_init<float>(I.Psi, I.T, N, K, problem->a_rad, problem->c, h->st)
                 : launch_sn_init<double>(I.Psi, I.T, N, K, problem->a_rad, problem->c, h->st);
  }
  chain(cudaStreamSynchronize(h->st));
  if (e != cudaSuccess) {
    std::string msg = cudaGetErrorString(e);
    cudaFreeHost(h->h_status);
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return fail(DLR_ECUDA, "upload failed: %s", msg.c_str());
  }
  *out = h;
  return DLR_OK;
}

int dlr_create(const dlr_problem *problem, const dlr_runtime *runtime, dlr_handle **out) {
  if (!out) return fail(DLR_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(problem);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(DLR_ECUDA, "no CUDA device");
  {
    // the kernels are built for sm_103a only: fail loudly on anything else
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_widen);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(DLR_ECUDA, "kernels cannot run on this GPU: %s", cudaGetErrorString(e));
    }
  }
  dlr_handle *h = new dlr_handle();
  h->prob = *problem;
  h->prob.sigma = h->prob.rho_cv = h->prob.T0 = nullptr;
  h->mixed = problem->precision == DLR_MIXED;
  h->rs = h->mixed ? 4 : 8;
  h->N = problem->nx * problem->ny;
  h->K = problem->n_polar * problem->n_azim;
  h->r = problem->rank;
  if (runtime) h->rt = *runtime;
  h->st = (cudaStream_t)h->rt.stream;
  if (!h->st) {  // graphs cannot be captured on the legacy stream
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return fail(DLR_ECUDA, "stream creation failed");
    }
    h->own_stream = true;
  }
  const Sizes sz = sizes_of(problem, num_sms());
  if (h->rt.hbm_budget && sz.total > h->rt.hbm_budget) {
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return fail(DLR_ENOMEM, "footprint %zu bytes exceeds the HBM budget %zu", sz.total, h->rt.hbm_budget);
  }
  h->pb = sz.pb;
  h->pbl = sz.pbl;
  h->lb = sz.lb;
  h->pbg = sz.pbg;
  build_quadrature(h);
  if (problem->method == DLR_METHOD_SN) return create_sn(h, problem, out);
  std::vector<double> X0, W0;
  double fn = 0.0;
  // bilinear elements: at most N DG0 modes, the rest of X0 on the slopes
  const int rx = problem->element == 1 ? std::min(h->r, h->N) : h->r;
  if (!build_W0(h, W0) || !build_X0(h, problem->T0, rx, X0, fn)) {
    delete h;
    return fail(DLR_EINVAL, "rank %d exceeds the independent initial basis functions", h->r);
  }
  const int N = h->N, K = h->K, r = h->r;
  const size_t rs = h->rs;
  Inst &I = h->inst;
  fill_common(h, problem);
  I.lay = small_layout(r);
  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = dev_alloc(h, bytes);
    ok = ok && p;
    return p;
  };
  double *sigma = (double *)A((size_t)N * 8);
  double *rho = (double *)A((size_t)N * 8);
  I.T = (double *)A((size_t)N * 8);
  I.B0 = (double *)A((size_t)N * 8);
  I.D = (double *)A((size_t)N * 8);
  I.sigma = sigma;
  I.rho_cv = rho;
  I.sig_t = A((size_t)N * rs);
  I.ss4 = A((size_t)N * rs);
  I.q = A((size_t)N * rs);
  I.phi0 = A((size_t)N * rs);
  I.phi1 = A((size_t)N * rs);
  I.sphi = A((size_t)N * rs);
  // the augmented step keeps X0, W0 with m = 2r columns (the last r zero
  // between steps) and runs steps 5-10 on a rank-2r copy of the instance
  const bool aug = problem->augment == 1;
  const int m = aug ? 2 * r : r;
  h->aug = aug;
  const size_t rowsN = I.q1 ? (size_t)4 * N : (size_t)N;  // rows of X (Q1: 4 per cell)
  if (I.q1) {
    I.phi0 = A(rowsN * rs);
    I.phi1 = A(rowsN * rs);
    I.q1_wt = (double *)A(rowsN * 8);
    I.q1_ws = (double *)A(rowsN * 8);
    I.q1_v = A(rowsN * r * rs);
  }
  I.X0 = A(rowsN * m * rs);
  I.X = A(rowsN * m * rs);
  I.Psi = A(rowsN * m * rs);
  I.s0 = A(rowsN * r * rs);
  double *dox = (double *)A((size_t)K * 8), *doy = (double *)A((size_t)K * 8), *dw = (double *)A((size_t)K * 8);
  I.ox = dox;
  I.oy = doy;
  I.w = dw;
  I.W0 = (double *)A((size_t)K * m * 8);
  I.L = (double *)A((size_t)K * m * 8);
  I.Lf = (double *)A((size_t)K * m * 8);
  I.S0 = (double *)A((size_t)r * r * 8);
  I.idx = (int *)A((size_t)r * 4);
  I.small = (double *)A((size_t)I.lay.total * 8);
  I.lu = (double *)A((size_t)K * m * m * 8);
  I.piv = (int *)A((size_t)K * m * 4);
  const SmallLayout lay2 = small_layout(m);
  double *S0m = aug ? (double *)A((size_t)m * m * 8) : nullptr;
  double *small2 = aug ? (double *)A((size_t)lay2.total * 8) : nullptr;
  I.partials = (double *)A(sz.partial_doubles * 8);
  I.partial_blocks = h->pb;
  I.angle_blocks = h->pbl;
  I.lstep_blocks = h->lb;
  I.status = (int *)A(64);
  I.nonpos = (int *)A(64);
  I.allow_nonpos = problem->allow_nonpositive ? 1 : 0;
  I.iters = (int *)A(64);
  I.conv = (unsigned long long *)A(64);
  h->d_iters_total = (long long *)A(64);
  I.iters_total = (unsigned long long *)h->d_iters_total;
  alloc_dsa(h, A);
  if (problem->reflect[0] || problem->reflect[1] || problem->reflect[2] || problem->reflect[3]) {
    const size_t LB = (size_t)problem->nx + problem->ny;
    I.refl_base = A((size_t)r * LB * rs);
    I.refl_kap = (double *)A(2 * LB * r * 8);
    I.refl_data = (double *)A((size_t)K * LB * 8);
    I.refl_y = (double *)A((size_t)K * r * 8);
    I.refl_u = (double *)A((size_t)K * r * 8);
    I.refl_passes = (int *)A(64);
  }
  I.grp = grp_eligible(problem) ? 1 : 0;
  I.grp_tab = nullptr;
  I.sgk = I.spk = I.part = I.qsum = nullptr;
  if (I.grp) {
    I.grp_ng = grp_count(r);
    I.nwin = grp_nwin(problem->nx);
    I.nbands = (problem->ny + 31) / 32;
    I.glay = grp_lay(problem->nx, problem->ny);
    I.grp_tab = (int *)A((size_t)I.grp_ng * kGrpRec * 4);
    I.sgk = (float *)A((size_t)I.grp_ng * (kGA + 1) * I.glay * 4);
    I.spk = (float *)A(8 * I.glay * 4);
    I.part = (float *)A((size_t)I.grp_ng * I.glay * 4);
    I.qsum = (float *)A(4 * I.glay * 4);
  }
  if (!ok) {
    dev_free_all(h);
    delete h;
    return fail(DLR_ENOMEM, "device allocation failed");
  }
  if (cudaMallocHost(&h->h_status, sizeof(int)) != cudaSuccess) {
    dev_free_all(h);
    delete h;
    return fail(DLR_ENOMEM, "pinned allocation failed");
  }
  *h->h_status = 0;
  // host -> device
  std::vector<double> S0(r * r, 0.0);
  S0[0] = fn * std::sqrt(4.0 * kPi);
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st);
  };
  cudaError_t e = cudaSuccess;
  auto chain = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chain(up(sigma, problem->sigma, (size_t)N * 8));
  chain(up(rho, problem->rho_cv, (size_t)N * 8));
  chain(up(I.T, problem->T0, (size_t)N * 8));
  chain(up(dox, h->ox.data(), (size_t)K * 8));
  chain(up(doy, h->oy.data(), (size_t)K * 8));
  chain(up(dw, h->w.data(), (size_t)K * 8));
  if (aug) {  // zero the extra columns of X0 and W0 (and the rank-2r work space)
    chain(cudaMemsetAsync(I.X0, 0, (size_t)N * m * rs, h->st));
    chain(cudaMemsetAsync(I.W0, 0, (size_t)K * m * 8, h->st));
    chain(cudaMemsetAsync(S0m, 0, (size_t)m * m * 8, h->st));
    chain(cudaMemsetAsync(small2, 0, (size_t)lay2.total * 8, h->st));
  }
  chain(up(I.W0, W0.data(), (size_t)K * r * 8));
  chain(up(I.S0, S0.data(), (size_t)r * r * 8));
  if (I.grp) {  // the padding of the skewed layouts stays zero
    chain(cudaMemsetAsync(I.sgk, 0, (size_t)I.grp_ng * (kGA + 1) * I.glay * 4, h->st));
    chain(cudaMemsetAsync(I.spk, 0, 8 * I.glay * 4, h->st));
  }
  std::vector<double> X0q;  // the Q1 basis (rows 4 c + m), uploaded in place of X0
  if (I.q1) {
    // the DG0 basis as Q1 fields: each cell's constant coefficient (stored
    // scale 1), slopes zero; still orthonormal in the h^2 inner product
    X0q.assign((size_t)4 * N * r, 0.0);
    for (int l = 0; l < rx; ++l)
      for (int c = 0; c < N; ++c) X0q[(size_t)4 * c + (size_t)4 * N * l] = X0[c + (size_t)N * l];
    // columns beyond the N cell constants (r > N on tiny meshes): one slope
    // coefficient each, scaled to unit h^2 norm (they carry no psi0)
    for (int l = rx; l < r; ++l) {
      const int q = l - rx, c = q / 3, m = 1 + q % 3;
      X0q[(size_t)4 * c + m + (size_t)4 * N * l] = 1.0 / std::sqrt(I.h2);
    }
  }
  const std::vector<double> &X0u = I.q1 ? X0q : X0;
  if (h->mixed) {
    std::vector<float> Xf(X0u.begin(), X0u.end());
    chain(up(I.X0, Xf.data(), Xf.size() * 4));
  } else {
    chain(up(I.X0, X0u.data(), X0u.size() * 8));
  }
  chain(cudaMemsetAsync(I.status, 0, 64, h->st));
  chain(cudaMemsetAsync(I.nonpos, 0, 64, h->st));
  chain(cudaMemsetAsync(I.iters, 0, 64, h->st));
  chain(cudaMemsetAsync(h->d_iters_total, 0, 64, h->st));
  if (h->d_dsa_iters_total) chain(cudaMemsetAsync(h->d_dsa_iters_total, 0, 64, h->st));
  chain(cudaMemsetAsync(I.idx, 0xff, (size_t)r * 4, h->st));
  chain(cudaMemsetAsync(I.small, 0, (size_t)I.lay.total * 8, h->st));
  if (I.refl_passes) chain(cudaMemsetAsync(I.refl_passes, 0, 64, h->st));
  // the host vectors above are released on return: wait for the copies
  chain(cudaStreamSynchronize(h->st));
  if (e != cudaSuccess) {
    std::string msg = cudaGetErrorString(e);
    cudaFreeHost(h->h_status);
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return fail(DLR_ECUDA, "upload failed: %s", msg.c_str());
  }
  if (aug) {
    // steps 1-4 sweep Psi into the first r columns of the step-5 input and
    // copy X0 beside it; steps 5-10 see the instance at rank m = 2r
    I.aug_x0 = static_cast<char *>(I.Psi) + (size_t)N * r * rs;
    Inst &J = h->inst2;
    J = I;
    J.r = m;
    J.lay = lay2;
    J.small = small2;
    J.S0 = S0m;
    J.aug_r = r;
    J.S0_r = I.S0;
    J.aug_x0 = nullptr;
  }
  *out = h;
  return DLR_OK;
}

void dlr_destroy(dlr_handle *h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  purge_batches(h);
  if (h->own_batch) destroy_batch(h->own_batch);
  for (auto &p : h->ev_pending)
    for (auto ev : p) cudaEventDestroy(ev);
  for (auto ev : h->ev_pool) cudaEventDestroy(ev);
  if (h->h_status) cudaFreeHost(h->h_status);
  dev_free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
}

// ------------------------------------------------------------------
// batch plans
// ------------------------------------------------------------------
static void destroy_batch(Batch *b) {
  if (!b) return;
  if (b->pre) cudaGraphExecDestroy(b->pre);
  if (b->post) cudaGraphExecDestroy(b->post);
  if (b->si) cudaGraphExecDestroy(b->si);
  if (b->d_mem) cudaFree(b->d_mem);
  delete b;
}

template <typename T>
static T *carve(char *&cur, size_t count) {
  T *p = reinterpret_cast<T *>(cur);
  cur += (count * sizeof(T) + 255) & ~size_t(255);
  return p;
}

// ------------------------------------------------------------------
// sweep work units and their autotuning
// ------------------------------------------------------------------

// Modelled wavefront steps of one unit of p bands (32 rows each) on an
// nx-column mesh swept by nw warps: each warp sweeps ceil(p / nw) bands one
// after the other, and the warps start one band lag apart (the 31-step skew
// of a band plus its progress granularity: `lag` steps).
static double unit_steps(int nx, int p, int nw, int lag) {
  return (double)((p + nw - 1) / nw) * (nx + 31) + (std::min(p, nw) - 1) * (double)lag;
}

// Splits angles into units of consecutive bands.  Starting from one unit per
// (instance, angle), the instance with the longest unit is split (bands per
// unit halved, kept a multiple of nw) while its unit takes longer than
// `split` times the average load of one of the `ctas` resident CTAs; split <= 0
// keeps one unit per angle.  Units are ordered by modelled length, longest
// first, and the units of one angle bottom-up, so that a unit's predecessor
// is always claimed before it.  Returns the number of edge rows used.
// Sweep items per instance: its r angles (per-angle kernel) or its groups
// of angles (grouped kernel; a unit's `angle` is then the group index).
static int sweep_items(const dlr_handle *h, bool grp) { return grp ? h->inst.grp_ng : h->r; }

static int plan_units(dlr_handle *const *hs, int n, bool mixed, bool grp, int ctas, double split,
                      std::vector<SiUnit> &units) {
  if (hs[0]->inst.q1) {  // the bilinear sweep takes a whole angle per unit
    units.clear();
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < hs[i]->r; ++j) units.push_back(SiUnit{i, j, 0, (hs[i]->prob.ny + 31) / 32, -1, -1});
    return (int)units.size();
  }
  const int nw = grp ? si_grp_warps() : si_sweep_warps(mixed);
  const int lag = grp ? si_grp_lag() : si_sweep_lag(mixed);
  std::vector<int> nb(n), bpu(n);
  for (int i = 0; i < n; ++i) bpu[i] = nb[i] = (hs[i]->prob.ny + 31) / 32;
  while (split > 0) {
    double total = 0, tmax = 0;
    int imax = -1;
    for (int i = 0; i < n; ++i) {
      const int g = (nb[i] + bpu[i] - 1) / bpu[i];
      const double t = unit_steps(hs[i]->prob.nx, bpu[i], nw, lag);
      total += (double)sweep_items(hs[i], grp) * g * t;
      if (bpu[i] > nw && t > tmax) {
        tmax = t;
        imax = i;
      }
    }
    if (imax < 0 || tmax <= split * total / ctas) break;
    const int half = (bpu[imax] + 1) / 2;
    bpu[imax] = std::max(nw, (half + nw - 1) / nw * nw);
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return unit_steps(hs[a]->prob.nx, bpu[a], nw, lag) > unit_steps(hs[c]->prob.nx, bpu[c], nw, lag);
  });
  units.clear();
  int rows = 0;
  for (int i : order) {
    const int g = (nb[i] + bpu[i] - 1) / bpu[i];
    for (int j = 0; j < sweep_items(hs[i], grp); ++j) {
      for (int q = 0; q < g; ++q) {
        SiUnit u;
        u.inst = i;
        u.angle = j;
        u.b0 = q * bpu[i];
        u.nb = std::min(bpu[i], nb[i] - q * bpu[i]);
        u.in_row = q > 0 ? rows + q - 1 : -1;
        u.out_row = q + 1 < g ? rows + q : -1;
        units.push_back(u);
      }
      rows += g - 1;
    }
  }
  return rows;
}

// Autotuned sweep plans by batch shape (the sorted (nx, ny, r, precision)
// of its instances): the splitting threshold and the source-iteration
// kernel (grouped: two angles per warp; or one angle per warp).
struct TunedPlan {
  double split;
  int grouped;
};
static std::map<std::vector<std::array<int, 4>>, TunedPlan> &tune_table() {
  static std::map<std::vector<std::array<int, 4>>, TunedPlan> m;
  return m;
}
static std::vector<std::array<int, 4>> batch_shape(dlr_handle *const *hs, int n);
constexpr double kDefaultSplit = 1.0;
// Untuned, the grouped kernel serves batches whose largest mesh has at least
// this many cells (measured: it is 1.3x faster per source iteration on
// 1024^2 cells, 1.3x slower on 256^2, and even on a batch of 64^2-512^2
// meshes).
constexpr long long kGroupedMinCells = 1ll << 19;

static TunedPlan tuned_plan(dlr_handle *const *hs, int n) {
  bool forced = true;  // sweep_mode 2 on every instance: the grouped kernel
  for (int i = 0; i < n; ++i) forced = forced && hs[i]->prob.sweep_mode == 2;
  auto &m = tune_table();
  auto it = m.find(batch_shape(hs, n));
  if (forced) return TunedPlan{it != m.end() ? it->second.split : kDefaultSplit, 1};
  if (it != m.end()) return it->second;
  long long cmax = 0;
  for (int i = 0; i < n; ++i) cmax = std::max(cmax, (long long)hs[i]->N);
  return TunedPlan{kDefaultSplit, cmax >= kGroupedMinCells ? 1 : 0};
}

static int build_batch(dlr_handle *const *hs, int n, Batch **out) {
  Batch *b = new Batch();
  b->hs.assign(hs, hs + n);
  for (int i = 0; i < n; ++i) b->versions.push_back(hs[i]->version);
  b->n = n;
  b->mixed = hs[0]->mixed;
  b->st = hs[0]->st;
  // the SVD of S every step for DEIM (its angles depend on the basis) and
  // at full angular rank (r = NOm) on DG0 cells: there the factors kept in
  // the CholeskyQR basis between steps lost the weighted orthonormality of
  // W enough for the source iteration to stop converging (a 12 x 10 mesh
  // with 8 angles, FP64, third step), while the SVD basis keeps it
  b->svd_mode = hs[0]->prob.selection == DLR_SEL_DEIM ? 1 : 0;
  for (int i = 0; i < n; ++i)
    if (!hs[i]->sn && !hs[i]->inst.q1 && hs[i]->r == hs[i]->K) b->svd_mode = 1;
  b->sn = hs[0]->sn;
  b->aug = hs[0]->aug;
  b->q1 = hs[0]->inst.q1 != 0;
  for (int i = 0; i < n; ++i) {
    const dlr_handle *h = hs[i];
    b->maxN = std::max(b->maxN, h->N);
    b->maxK = std::max(b->maxK, h->K);
    b->rmax = std::max(b->rmax, h->aug ? 2 * h->r : h->r);  // rank of steps 5-10
    b->rmask |= rank_mask(h->aug ? 2 * h->r : h->r);
    b->rmask_pre |= rank_mask(h->r);
    b->pbmax = std::max(b->pbmax, h->pb);
    b->pbgmax = std::max(b->pbgmax, h->pbg);
    b->pblmax = std::max(b->pblmax, h->pbl);
    b->lbmax = std::max(b->lbmax, h->lb);
    b->nx_max = std::max(b->nx_max, h->prob.nx);
    b->maxL = std::max(b->maxL, h->prob.nx + h->prob.ny);
    b->maxRows = std::max(b->maxRows, h->inst.q1 ? 4 * h->N : h->N);
    b->refl = b->refl || h->inst.refl_kap != nullptr;
    b->bands_max = std::max(b->bands_max, (h->prob.ny + 31) / 32);
  }
  const int gam_max = b->sn ? b->rmax : kMaxRank;  // scalar-flux weights of k_si
  int any_dsa = 0;
  b->grp_ok = true;
  for (int i = 0; i < n; ++i) {
    any_dsa |= hs[i]->inst.dsa ? 1 : 0;
    b->grp_ok = b->grp_ok && hs[i]->inst.grp;
  }
  if (b->grp_ok) {
    b->grp_stages = si_grp_stages(b->nx_max, b->bands_max, n);
    if (b->grp_stages == 0) b->grp_ok = false;  // too wide for its shared memory: the per-angle kernel
  }
  b->grid_angle = b->mixed ? si_max_grid<float>(b->nx_max, b->bands_max, n, gam_max, any_dsa)
                           : si_max_grid<double>(b->nx_max, b->bands_max, n, gam_max, any_dsa);
  b->grid_grp = b->grp_ok ? si_grp_max_grid(b->nx_max, b->bands_max, n, b->grp_stages) : 0;
  if (b->grp_ok && b->grid_grp <= 0) b->grp_ok = false;
  if (b->q1)
    b->grid_angle = b->mixed ? q1_si_max_grid<float>(b->nx_max, b->bands_max, n, gam_max)
                             : q1_si_max_grid<double>(b->nx_max, b->bands_max, n, gam_max);
  if (b->grid_angle <= 0) {
    delete b;
    return fail(DLR_ECUDA, "the source-iteration kernel does not fit on this GPU");
  }
  const TunedPlan tp = tuned_plan(hs, n);
  b->grp = b->grp_ok && tp.grouped;
  b->si_grid = b->grp ? b->grid_grp : b->grid_angle;
  const int gmax = b->si_grid;
  // capacity of the unit and edge tables: the finest split (one unit per
  // NW bands, or per band when an angle has fewer bands than warps), for
  // either kernel
  int rows_cap = 0;
  for (int kind = 0; kind < (b->grp_ok ? 2 : 1); ++kind) {
    const bool g1 = kind == 1;
    const int nw = g1 ? si_grp_warps() : si_sweep_warps(b->mixed);
    int units = 0, rows = 0;
    for (int i = 0; i < n; ++i) {
      const int nb = (hs[i]->prob.ny + 31) / 32;
      const int g = (nb + std::min(nb, nw) - 1) / std::min(nb, nw);
      units += sweep_items(hs[i], g1) * g;
      rows += sweep_items(hs[i], g1) * (g - 1);
    }
    b->units_cap = std::max(b->units_cap, units);
    rows_cap = std::max(rows_cap, rows);
  }
  b->split = tp.split;
  std::vector<SiUnit> units;
  plan_units(hs, n, b->mixed, b->grp, gmax, b->split, units);
  // one device block for the batch's tables
  size_t bytes = 0;
  auto sz = [](size_t s) { return (s + 255) & ~size_t(255); };
  bytes += 2 * sz(sizeof(Inst) * n);
  bytes += 9 * sz(sizeof(GramJob) * n) + 2 * sz(sizeof(FillJob) * n) + 9 * sz(sizeof(ApplyJob) * n) +
           8 * sz(sizeof(CholJob) * n) + sz(sizeof(ReduceJob) * n);
  bytes += sz(sizeof(GramJob) * 7 * n) + sz(sizeof(ReduceJob) * 7 * n);  // bilinear elements
  // 64-bit words per edge row: one per column and value (two per FP64 value;
  // kGA values per column in the grouped sweep)
  const int gedge_ld = (b->nx_max + 3) / 4 * 4 * (b->grp_ok ? kGA : b->mixed ? 1 : 2);
  bytes += sz(sizeof(SiUnit) * b->units_cap) + sz(64) * 4;
  // one row more than any plan uses: zeroed below and never written (tags
  // are nonzero), the row dlr_debug_lose_edge points a unit at
  bytes += sz(sizeof(unsigned long long) * gedge_ld * (rows_cap + 1));
  const size_t dsa_part = any_dsa ? (size_t)n * kDsaSlots * gmax : 0;  // per-CTA CG partials
  bytes += sz(sizeof(double) * std::max<size_t>(1, dsa_part));
  bytes += sz(sizeof(GrpSi)) + 2 * sz(sizeof(int) * n) + sz(sizeof(double) * 3 * n);  // loop state of the grouped sweep
  if (cudaMalloc(&b->d_mem, bytes) != cudaSuccess) {
    delete b;
    return fail(DLR_ENOMEM, "batch table allocation failed");
  }
  // zeroed once: the launch counter, and edge words that can never carry a
  // valid tag (tags are nonzero)
  if (cudaMemsetAsync(b->d_mem, 0, bytes, hs[0]->st) != cudaSuccess) {
    cudaFree(b->d_mem);
    delete b;
    return fail(DLR_ECUDA, "batch table initialisation failed");
  }
  char *cur = (char *)b->d_mem;
  b->d_insts = carve<Inst>(cur, n);
  b->d_insts2 = carve<Inst>(cur, n);
  b->g_psi1 = carve<GramJob>(cur, n);
  b->g_psire = carve<GramJob>(cur, n);
  b->g_x = carve<GramJob>(cur, n);
  b->g_x3 = carve<GramJob>(cur, n);
  b->g_l1 = carve<GramJob>(cur, n);
  b->g_lf = carve<GramJob>(cur, n);
  b->g_w = carve<GramJob>(cur, n);
  b->g_w3 = carve<GramJob>(cur, n);
  b->g_cross = carve<GramJob>(cur, n);
  b->f_psi = carve<FillJob>(cur, n);
  b->f_l = carve<FillJob>(cur, n);
  b->a_psi = carve<ApplyJob>(cur, n);
  b->a_x2 = carve<ApplyJob>(cur, n);
  b->a_x3 = carve<ApplyJob>(cur, n);
  b->a_l1 = carve<ApplyJob>(cur, n);
  b->a_w2 = carve<ApplyJob>(cur, n);
  b->a_w3 = carve<ApplyJob>(cur, n);
  b->a_wv = carve<ApplyJob>(cur, n);
  b->a_cw = carve<ApplyJob>(cur, n);
  b->a_cx = carve<ApplyJob>(cur, n);
  b->c_p1 = carve<CholJob>(cur, n);
  b->c_p1b = carve<CholJob>(cur, n);
  b->c_p2 = carve<CholJob>(cur, n);
  b->c_p3 = carve<CholJob>(cur, n);
  b->c_l1 = carve<CholJob>(cur, n);
  b->c_l1b = carve<CholJob>(cur, n);
  b->c_l2 = carve<CholJob>(cur, n);
  b->c_l3 = carve<CholJob>(cur, n);
  b->r_proj = carve<ReduceJob>(cur, n);
  b->g_q1t = carve<GramJob>(cur, 7 * n);
  b->r_q1 = carve<ReduceJob>(cur, 7 * n);
  b->d_units = carve<SiUnit>(cur, b->units_cap);
  b->ctl.bar = carve<unsigned>(cur, 16);
  b->ctl.work = carve<unsigned>(cur, 16);
  b->ctl.abort_flag = carve<int>(cur, 16);
  b->ctl.epoch = carve<unsigned>(cur, 16);
  b->ctl.gedge = carve<unsigned long long>(cur, (size_t)gedge_ld * (rows_cap + 1));
  b->ctl.n_rows = rows_cap;
  b->spare_row = rows_cap;
  b->ctl.gedge_ld = gedge_ld;
  b->ctl.dsa_part = carve<double>(cur, std::max<size_t>(1, dsa_part));
  b->ctl.any_dsa = any_dsa;
  b->ctl.force_iters = 0;
  b->ctl.units = b->d_units;
  b->ctl.n_units = (int)units.size();
  b->gs = carve<GrpSi>(cur, 1);
  {
    GrpSi g{};
    g.n_units = b->ctl.n_units;
    g.active = carve<int>(cur, n);
    g.par_of = carve<int>(cur, n);
    g.relax = carve<double>(cur, 3 * n);
    if (cudaMemcpyAsync(b->gs, &g, sizeof g, cudaMemcpyHostToDevice, hs[0]->st) != cudaSuccess ||
        cudaStreamSynchronize(hs[0]->st) != cudaSuccess) {
      cudaFree(b->d_mem);
      delete b;
      return fail(DLR_ECUDA, "batch table initialisation failed");
    }
  }
  b->ctl.n_inst = n;
  b->ctl.nx_max = b->nx_max;
  b->ctl.bands_max = b->bands_max;
  b->ctl.gam_max = gam_max;
  // host copies of the job tables
  std::vector<Inst> insts(n), insts2(n);
  std::vector<GramJob> gp1(n), gpre(n), gx(n), gx3(n), gl1(n), glf(n), gw(n), gw3(n), gcr(n);
  std::vector<FillJob> fp(n), fl(n);
  std::vector<ApplyJob> ap(n), ax2(n), ax3(n), al1(n), aw2(n), aw3(n), awv(n), acw(n), acx(n);
  std::vector<CholJob> cp1(n), cp1b(n), cp2(n), cp3(n), cl1(n), cl1b(n), cl2(n), cl3(n);
  std::vector<ReduceJob> rp(n);
  std::vector<GramJob> gq(7 * n);
  std::vector<ReduceJob> rq(7 * n);
  for (int i = 0; i < n; ++i) {
    const dlr_handle *h = hs[i];
    insts[i] = h->inst;
    insts2[i] = h->aug ? h->inst2 : h->inst;
    if (b->sn) continue;  // the SN step uses no job tables
    // the jobs of steps 5-10 (rank 2r when augmented)
    const Inst &I = insts2[i];
    const int N = h->N, K = h->K, r = I.r;
    double *sm = I.small;
    const SmallLayout &L = I.lay;
    int *flag = reinterpret_cast<int *>(sm + L.qr_flag);
    auto gram = [&](const void *A, const double *wt, int m, int lda, int layout, int nb, const int *run_if) {
      GramJob g{};
      g.A = A; g.wt = wt; g.m = m; g.r = r; g.lda = lda; g.layout = layout;
      g.out = I.partials; g.nblocks = nb; g.run_if = run_if;
      return g;
    };
    // the Grams of step 5: k_gram32 in mixed precision, k_tsgram in FP64
    // (one partial per cluster either way)
    const int pbx = h->mixed ? h->pbg : h->pb;
    const int NR = I.q1 ? 4 * N : N;  // rows of Psi and X (Q1: 4 coefficients per cell)
    gp1[i] = gram(I.Psi, nullptr, NR, NR, 0, pbx, nullptr);
    gpre[i] = gram(I.Psi, nullptr, NR, NR, 0, pbx, flag + 1);
    gx[i] = gram(I.X, nullptr, NR, NR, 0, pbx, nullptr);
    gl1[i] = gram(I.L, I.w, K, r, 1, h->pbl, nullptr);
    glf[i] = gram(I.Lf, I.w, K, r, 1, h->pbl, flag + 1);
    gw[i] = gram(I.W0, nullptr, K, K, 0, h->pbl, nullptr);
    gcr[i] = gram(I.L, I.w, K, r, 1, h->pbl, nullptr);
    gcr[i].B = I.W0;
    gcr[i].ldb = K;
    gcr[i].sqrt_wt = 1;
    // the third-pass Grams run only when the first passes were shifted
    gx3[i] = gram(I.X, nullptr, NR, NR, 0, pbx, flag);
    gw3[i] = gram(I.W0, nullptr, K, K, 0, h->pbl, flag);
    auto fill = [&](void *A, const void *src, int m, int lda, int layout) {
      FillJob f{};
      f.A = A; f.src = src; f.m = m; f.r = r; f.lda = lda; f.layout = layout; f.flag = flag;
      return f;
    };
    fp[i] = fill(I.Psi, nullptr, NR, NR, 0);
    fl[i] = fill(I.Lf, I.L, K, r, 1);
    auto apply = [&](const void *A, int layout, int lda, const double *s_in, int sq_in, const double *T,
                     void *outp, int ldo, const double *s_out, int inv_sq, int m, const int *run_if) {
      ApplyJob a{};
      a.A = A; a.in_layout = layout; a.lda = lda; a.s_in = s_in; a.sq_in = sq_in; a.T = T;
      a.out = outp; a.ldo = ldo; a.s_out = s_out; a.inv_sq_out = inv_sq; a.m = m; a.r = r;
      a.run_if = run_if;
      return a;
    };
    // CholeskyQR passes: Q = A R^{-1} by forward substitution
    auto solve = [&](const void *A, int layout, int lda, const double *s_in, const double *R,
                     void *outp, int ldo, int m, const int *run_if) {
      ApplyJob a = apply(A, layout, lda, s_in, s_in ? 1 : 0, R, outp, ldo, nullptr, 0, m, run_if);
      a.tri = 1;
      return a;
    };
    ap[i] = solve(I.Psi, 0, NR, nullptr, sm + L.R1, I.X, NR, NR, nullptr);
    ax2[i] = solve(I.X, 0, NR, nullptr, sm + L.R2, I.X, NR, NR, nullptr);
    ax3[i] = solve(I.X, 0, NR, nullptr, sm + L.R3, I.X, NR, NR, flag);
    al1[i] = solve(I.Lf, 1, r, I.w, sm + L.R1, I.W0, K, K, nullptr);
    aw2[i] = solve(I.W0, 0, K, nullptr, sm + L.R2, I.W0, K, K, nullptr);
    aw3[i] = solve(I.W0, 0, K, nullptr, sm + L.R3, I.W0, K, K, flag);
    awv[i] = apply(I.W0, 0, K, nullptr, 0, sm + L.V, I.W0, K, I.w, 1, K, nullptr);
    acw[i] = apply(I.W0, 0, K, nullptr, 0, sm + L.V, I.W0, K, nullptr, 0, K, nullptr);
    acx[i] = apply(I.X0, 0, NR, nullptr, 0, sm + L.U, I.X0, NR, nullptr, 0, NR, nullptr);
    const double u = chol_u(h->mixed), tau = chol_tau(h->mixed);
    auto chol = [&](int nparts, double scale, double *R, int mode) {
      CholJob c{};
      c.part = I.partials; c.nblocks = nparts; c.scale = scale; c.R = R;
      c.flag = flag; c.r = r; c.mode = mode; c.u = u; c.tau_dep = tau;
      return c;
    };
    const int pc = h->pb / kCl, pcl = h->pbl / kCl;  // partials: one per cluster
    const int pcx = h->mixed ? h->pbg / kCl : pc;      // (k_gram32 in mixed precision)
    cp1[i] = chol(pcx, I.h2, sm + L.R1, 1);
    cp1b[i] = chol(pcx, I.h2, sm + L.R1, 4);
    cp2[i] = chol(pcx, I.h2, sm + L.R2, 2);
    cp3[i] = chol(pcx, I.h2, sm + L.R3, 3);
    cl1[i] = chol(pcl, 1.0, sm + L.R1, 1);
    cl1b[i] = chol(pcl, 1.0, sm + L.R1, 4);
    cl2[i] = chol(pcl, 1.0, sm + L.R2, 2);
    cl3[i] = chol(pcl, 1.0, sm + L.R3, 3);
    ReduceJob red{};
    // (mixed DG0: one partial per CTA of k_project_tc5; else one per cluster)
    red.part = I.partials; red.nblocks = h->mixed && !I.q1 ? h->pb : pc; red.stride = proj_count(r);
    red.count = proj_count(r); red.out = sm + L.G; red.scale = 1.0;
    rp[i] = red;
    if (I.q1) {
      // step 7 on bilinear elements: A_x+, A_x-, A_y+, A_y- = X^T (T X)
      // (cross Grams with the transport buffer, filled one direction at a
      // time), M_t, M_s (row weights sigma_t, sigma_s) and P = <X, X0>, each
      // into its own block of partials, then reduced into the small slots
      const int slots[7] = {L.Axp, L.Axm, L.Ayp, L.Aym, L.Mt, L.Ms, L.P};
      for (int g = 0; g < 7; ++g) {
        double *part = I.partials + (size_t)g * pc * r * r;
        GramJob q = gram(I.X, nullptr, NR, NR, 0, h->pb, nullptr);
        q.out = part;
        if (g < 4) { q.B = I.q1_v; q.ldb = NR; }
        if (g == 4) q.wt = I.q1_wt;
        if (g == 5) q.wt = I.q1_ws;
        if (g == 6) { q.B = I.X0; q.ldb = NR; }
        gq[(size_t)g * n + i] = q;
        ReduceJob rj{};
        rj.part = part; rj.nblocks = pc; rj.stride = r * r; rj.count = r * r;
        rj.out = sm + slots[g]; rj.scale = g < 4 ? 1.0 : I.h2;
        rq[(size_t)g * n + i] = rj;
      }
    }
  }
  auto upv = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  auto chain = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  cudaStreamSynchronize(b->st);
  chain(upv(b->d_insts, insts.data(), sizeof(Inst) * n));
  chain(upv(b->d_insts2, insts2.data(), sizeof(Inst) * n));
  chain(upv(b->g_psi1, gp1.data(), sizeof(GramJob) * n));
  chain(upv(b->g_psire, gpre.data(), sizeof(GramJob) * n));
  chain(upv(b->g_x, gx.data(), sizeof(GramJob) * n));
  chain(upv(b->g_x3, gx3.data(), sizeof(GramJob) * n));
  chain(upv(b->g_l1, gl1.data(), sizeof(GramJob) * n));
  chain(upv(b->g_lf, glf.data(), sizeof(GramJob) * n));
  chain(upv(b->g_w, gw.data(), sizeof(GramJob) * n));
  chain(upv(b->g_w3, gw3.data(), sizeof(GramJob) * n));
  chain(upv(b->g_cross, gcr.data(), sizeof(GramJob) * n));
  chain(upv(b->f_psi, fp.data(), sizeof(FillJob) * n));
  chain(upv(b->f_l, fl.data(), sizeof(FillJob) * n));
  chain(upv(b->a_psi, ap.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_x2, ax2.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_x3, ax3.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_l1, al1.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_w2, aw2.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_w3, aw3.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_wv, awv.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_cw, acw.data(), sizeof(ApplyJob) * n));
  chain(upv(b->a_cx, acx.data(), sizeof(ApplyJob) * n));
  chain(upv(b->c_p1, cp1.data(), sizeof(CholJob) * n));
  chain(upv(b->c_p1b, cp1b.data(), sizeof(CholJob) * n));
  chain(upv(b->c_p2, cp2.data(), sizeof(CholJob) * n));
  chain(upv(b->c_p3, cp3.data(), sizeof(CholJob) * n));
  chain(upv(b->c_l1, cl1.data(), sizeof(CholJob) * n));
  chain(upv(b->c_l1b, cl1b.data(), sizeof(CholJob) * n));
  chain(upv(b->c_l2, cl2.data(), sizeof(CholJob) * n));
  chain(upv(b->c_l3, cl3.data(), sizeof(CholJob) * n));
  chain(upv(b->r_proj, rp.data(), sizeof(ReduceJob) * n));
  chain(upv(b->g_q1t, gq.data(), sizeof(GramJob) * 7 * n));
  chain(upv(b->r_q1, rq.data(), sizeof(ReduceJob) * 7 * n));
  chain(upv(b->d_units, units.data(), sizeof(SiUnit) * units.size()));
  // angle selection: one cluster of kCl CTAs per instance
  b->sel_slice_max = std::max(1, (b->maxK + kCl - 1) / kCl);
  // step 8 in one cluster kernel when the angles fit its shared memory
  b->lside_fused = b->svd_mode == 0 && b->maxK <= lside_max_k();
  if (e != cudaSuccess) {
    destroy_batch(b);
    return fail(DLR_ECUDA, "batch table upload failed: %s", cudaGetErrorString(e));
  }
  if (!b->sn && ((e = prepare_small(b->sel_slice_max, b->maxK, b->rmax)) != cudaSuccess ||
                  (e = prepare_dense(b->rmax)) != cudaSuccess ||
                  (b->lside_fused && (e = prepare_lside(b->sel_slice_max, b->rmax)) != cudaSuccess))) {
    destroy_batch(b);
    return fail(DLR_ECUDA, "kernel attribute setup failed: %s", cudaGetErrorString(e));
  }
  *out = b;
  return DLR_OK;
}

// refresh the batch's instance copies of handles changed since the upload
// (pageable sources are consumed before cudaMemcpyAsync returns)
static int refresh_batch(Batch *b) {
  for (int i = 0; i < b->n; ++i)
    if (b->versions[i] != b->hs[i]->version) {
      CK(cudaMemcpyAsync(b->d_insts + i, &b->hs[i]->inst, sizeof(Inst), cudaMemcpyHostToDevice, b->st));
      const Inst *j2 = b->hs[i]->aug ? &b->hs[i]->inst2 : &b->hs[i]->inst;
      CK(cudaMemcpyAsync(b->d_insts2 + i, j2, sizeof(Inst), cudaMemcpyHostToDevice, b->st));
      b->versions[i] = b->hs[i]->version;
    }
  return DLR_OK;
}

#define LK(call) \
  do {             \
    CK(call);      \
    ++b->kcount;   \
  } while (0)
// a launcher that launches one kernel per rank class in mask
#define LKM(call, mask)                      \
  do {                                       \
    CK(call);                                \
    b->kcount += __builtin_popcount(mask);   \
  } while (0)

template <typename real>
static int enqueue_pre(Batch *b) {
  const Inst *d = b->d_insts;
  const int n = b->n;
  if (b->sn) {  // full-rank SN: coefficients, fixed sources, starting phi
    if (b->q1) LK(launch_q1_coeff<real>(d, n, b->maxN, true, b->st));
    else LK(launch_sn_prep<real>(d, n, b->maxN, b->st));
    LK(launch_si_prep(d, n, b->ctl, b->st));
    return DLR_OK;
  }
  LK(launch_select(d, n, b->sel_slice_max, b->st));
  if (b->q1) {  // bilinear elements: coefficients, psi0, fixed sources, starting phi
    LK(launch_q1_coeff<real>(d, n, b->maxN, false, b->st));
    LK(launch_si_prep(d, n, b->ctl, b->st));
    return DLR_OK;
  }
  LKM(launch_coeff_recon<real>(d, n, b->maxN, b->rmask_pre, b->grp ? 1 : 0, b->st), b->rmask_pre);
  if (b->refl) {  // reflective edges: G, H and the first sweeps' inflow (two kernels)
    LK(launch_refl_pre<real>(d, n, b->rmax, b->maxL, b->st));
    ++b->kcount;
  }
  if (b->grp) LK(launch_grp_prep(d, n, b->ctl, b->gs, b->st));
  else LK(launch_si_prep(d, n, b->ctl, b->st));
  return DLR_OK;
}

template <typename real>
static int enqueue_post(Batch *b) {
  const Inst *d = b->d_insts2;  // steps 5-10 (rank 2r when augmented)
  const int n = b->n;
  cudaStream_t st = b->st;
  if (b->sn) {
    if (b->q1) LK(launch_q1_tupdate<real>(d, n, b->maxN, true, st));
    else LK(launch_sn_tupdate<real>(d, n, b->maxN, st));
    return DLR_OK;
  }
  // step 5: CholeskyQR of Psi; dependent columns are replaced by
  // pseudo-random ones (orthonormal completion) and the pass redone; a third
  // pass runs when a Cholesky needed a shift.  The augmented step factors
  // [Psi, X0] at rank 2r against the old factors padded to 2r columns.
  if (b->aug) LK(launch_aug_pad(d, n, st));
  if (b->refl) LK(launch_refl_kap<real>(d, n, b->rmax, b->maxL, st));  // What^-1 Psi at reflective edges
  // Grams of step 5 (FP32: k_gram32)
  auto gram5 = [&](const GramJob *g) {
    return b->mixed ? launch_gram32(g, n, b->pbgmax, st) : launch_tsgram<real>(g, n, b->pbmax, 0, st);
  };
  LK(gram5(b->g_psi1));
  LK(launch_chol(b->c_p1, d, n, st));
  LK(launch_fill<real>(b->f_psi, n, b->maxRows, st));
  LK(gram5(b->g_psire));
  LK(launch_chol(b->c_p1b, d, n, st));
  LKM((launch_apply<real, real>(b->a_psi, n, b->maxRows, b->rmask, st)), b->rmask);
  LK(gram5(b->g_x));
  LK(launch_chol(b->c_p2, d, n, st));
  LKM((launch_apply<real, real>(b->a_x2, n, b->maxRows, b->rmask, st)), b->rmask);
  LK(gram5(b->g_x3));
  LK(launch_chol(b->c_p3, d, n, st));
  LKM((launch_apply<real, real>(b->a_x3, n, b->maxRows, b->rmask, st)), b->rmask);
  // steps 6-7: projections and the L-step
  if (b->q1) {
    // bilinear elements: X^T (T X) per axis direction (the transport buffer
    // refilled for each), M_t, M_s, P, the seven reductions, q^, the edge
    // vectors and P S0
    for (int dir = 0; dir < 4; ++dir) {
      LK(launch_q1_transport<real>(d, n, b->maxN, dir, st));
      LK(launch_tsgram<real>(b->g_q1t + (size_t)dir * n, n, b->pbmax, 0, st));
    }
    LK(launch_tsgram<real>(b->g_q1t + (size_t)4 * n, 3 * n, b->pbmax, 0, st));
    LK(launch_reduce(b->r_q1, 7 * n, b->rmax * b->rmax, st));
    LK(launch_q1_vec<real>(d, n, b->pbmax, st));
    ++b->kcount;  // two kernels
  } else {
    // mixed precision: the tensor-core kernel, one launch per rank class
    LKM(launch_project<real>(d, n, b->pbmax, b->rmax, b->rmask, st), sizeof(real) == 4 ? b->rmask : 1);
    LK(launch_reduce(b->r_proj, n, proj_count(b->rmax), st));
    LK(launch_proj_post(d, n, st));
  }
  LKM(launch_lstep(d, n, b->rmax, b->rmask, b->lbmax, b->maxK, st), b->rmask);
  b->kcount += 2;  // and two more kernels
  if (b->refl) LK(launch_refl_lstep<real>(d, n, st));  // the reflected inflow's fixed point
  // step 8: CholeskyQR of M = diag(sqrt w) L^T into Q (held in W0), S = M^T Q,
  // SVD of S, W0 <- diag(1/sqrt w) Q V
  if (b->lside_fused) {
    LK(launch_lside(d, n, b->sel_slice_max, b->rmax, st));
  } else {
    LK(launch_tsgram<double>(b->g_l1, n, b->pblmax, 1, st));
    LK(launch_chol(b->c_l1, d, n, st));
    LK(launch_fill<double>(b->f_l, n, b->maxK, st));
    LK(launch_tsgram<double>(b->g_lf, n, b->pblmax, 1, st));
    LK(launch_chol(b->c_l1b, d, n, st));
    LKM((launch_apply<double, double>(b->a_l1, n, b->maxK, b->rmask, st)), b->rmask);
    LK(launch_tsgram<double>(b->g_w, n, b->pblmax, 0, st));
    LK(launch_chol(b->c_l2, d, n, st));
    LKM((launch_apply<double, double>(b->a_w2, n, b->maxK, b->rmask, st)), b->rmask);
    LK(launch_tsgram<double>(b->g_w3, n, b->pblmax, 0, st));
    LK(launch_chol(b->c_l3, d, n, st));
    LKM((launch_apply<double, double>(b->a_w3, n, b->maxK, b->rmask, st)), b->rmask);
    LK(launch_tsgram<double>(b->g_cross, n, b->pblmax, 1, st));
    LK(launch_svd(d, n, b->svd_mode, st));
    LKM((launch_apply<double, double>(b->a_wv, n, b->maxK, b->rmask, st)), b->rmask);
    if (b->svd_mode == 1) LK(launch_sign(d, n, b->maxK, st));
  }
  if (b->aug) {
    // SVD of the 2r x 2r S, truncation to the r largest singular values,
    // W0 <- W V (the last r columns zero); X0 <- X^ U in step 9
    LK(launch_svd(d, n, 2, st));
    LK(launch_aug_trunc(d, n, st));
    LKM((launch_apply<double, double>(b->a_cw, n, b->maxK, b->rmask, st)), b->rmask);
  }
  // step 9
  if (b->q1) LK(launch_q1_tupdate<real>(d, n, b->maxN, false, st));
  else LKM(launch_tupdate<real>(d, n, b->maxN, b->rmask, st), b->rmask);
  return DLR_OK;
}

static int capture(Batch *b, bool pre, cudaGraphExec_t *exec) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  int rc = pre ? (b->mixed ? enqueue_pre<float>(b) : enqueue_pre<double>(b))
               : (b->mixed ? enqueue_post<float>(b) : enqueue_post<double>(b));
  cudaError_t e = cudaStreamEndCapture(b->st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(DLR_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(DLR_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return DLR_OK;
}

static cudaEvent_t pool_event(dlr_handle *h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// The grouped source iteration as a graph: a while node whose body is one
// iteration (sweeps, quadrant sums, scalar flux and decision; the decision
// kernel ends the loop) and, after it, the last sweep that writes Psi.
static int capture_si(Batch *b) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle loop;
  cudaError_t e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNode_t wn = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(b->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e1 = launch_grp_iteration(b->d_insts, b->n, b->ctl, b->gs, b->si_grid, b->grp_stages,
                                              loop, b->st);
        e = cudaStreamEndCapture(b->st, &body);
        if (e == cudaSuccess) e = e1;
      }
    }
  }
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(b->st, g, &wn, nullptr, 1, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = launch_grp_final(b->d_insts, b->ctl, b->gs, b->si_grid, b->grp_stages, b->st);
      e = cudaStreamEndCapture(b->st, &g);
      if (e == cudaSuccess) e = e1;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->si, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(DLR_ECUDA, "source-iteration graph: %s", cudaGetErrorString(e));
  }
  return DLR_OK;
}

// The source-iteration launch of the batch with control block c (for the
// grouped sweep: its graph, after the loop state's forced iteration count
// is set to c.force_iters).
static cudaError_t launch_si_batch(const Batch *b, const SiCtl &c) {
  if (b->grp) {
    cudaError_t e = cudaMemcpyAsync(&b->gs->force_iters, &c.force_iters, sizeof(int), cudaMemcpyHostToDevice,
                                    b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&b->gs->n_units, &c.n_units, sizeof(int), cudaMemcpyHostToDevice,
                                              b->st);
    return e == cudaSuccess ? cudaGraphLaunch(b->si, b->st) : e;
  }
  if (b->q1)
    return b->mixed ? launch_q1_si<float>(b->d_insts, c, b->si_grid, b->st)
                    : launch_q1_si<double>(b->d_insts, c, b->si_grid, b->st);
  return b->mixed ? launch_si<float>(b->d_insts, c, b->si_grid, b->st)
                  : launch_si<double>(b->d_insts, c, b->si_grid, b->st);
}

static int ensure_graphs(Batch *b);

static int run_steps(Batch *b, int nsteps) {
  int rc = refresh_batch(b);
  if (rc) return rc;
  if ((rc = ensure_graphs(b))) return rc;
  dlr_handle *h0 = b->hs[0];
  for (int s = 0; s < nsteps; ++s) {
    std::array<cudaEvent_t, 4> ev{};
    const bool timing = h0->timing && b->n == 1;
    if (timing) {
      for (auto &x : ev) x = pool_event(h0);
      CK(cudaEventRecord(ev[0], b->st));
    }
    CK(cudaGraphLaunch(b->pre, b->st));
    if (timing) CK(cudaEventRecord(ev[1], b->st));
    CK(b->grp ? cudaGraphLaunch(b->si, b->st) : launch_si_batch(b, b->ctl));
    if (timing) CK(cudaEventRecord(ev[2], b->st));
    CK(cudaGraphLaunch(b->post, b->st));
    if (timing) {
      CK(cudaEventRecord(ev[3], b->st));
      h0->ev_pending.push_back(ev);
    }
  }
  for (auto *h : b->hs) {
    h->steps += nsteps;
    h->grp_loop = b->grp;
    h->canonical = b->svd_mode == 1 || b->aug;  // the augmented step ends on the SVD of S
    h->kernel_launches += (int64_t)nsteps * b->kernels_per_step;
    CK(cudaMemcpyAsync(h->h_status, h->inst.status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  }
  return DLR_OK;
}

int dlr_step(dlr_handle *h, int32_t nsteps) {
  if (!h) return fail(DLR_EINVAL, "handle is NULL");
  return dlr_step_batch(&h, 1, nsteps);
}

static std::map<std::vector<dlr_handle *>, Batch *> &batch_cache() {
  static std::map<std::vector<dlr_handle *>, Batch *> m;
  return m;
}

static void purge_batches(dlr_handle *h) {
  auto &m = batch_cache();
  for (auto it = m.begin(); it != m.end();) {
    if (std::find(it->first.begin(), it->first.end(), h) != it->first.end()) {
      destroy_batch(it->second);
      it = m.erase(it);
    } else {
      ++it;
    }
  }
}

static std::vector<std::array<int, 4>> batch_shape(dlr_handle *const *hs, int n) {
  std::vector<std::array<int, 4>> v;
  for (int i = 0; i < n; ++i)
    v.push_back({hs[i]->prob.nx, hs[i]->prob.ny, hs[i]->r, hs[i]->mixed ? 1 : 0});
  std::sort(v.begin(), v.end());
  return v;
}

static int check_handles(dlr_handle *const *hs, int n) {
  if (!hs || n < 1) return fail(DLR_EINVAL, "no handles");
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(DLR_EINVAL, "handle %d is NULL", i);
    if (hs[i]->mixed != hs[0]->mixed) return fail(DLR_EINVAL, "mixed precisions in one batch");
    if (hs[i]->st != hs[0]->st) return fail(DLR_EINVAL, "handles on different streams");
    if (hs[i]->sn != hs[0]->sn) return fail(DLR_EINVAL, "SN and DLR handles in one batch");
    if (hs[i]->aug != hs[0]->aug) return fail(DLR_EINVAL, "augmented and plain handles in one batch");
    if (hs[i]->inst.q1 != hs[0]->inst.q1) return fail(DLR_EINVAL, "DG0 and bilinear handles in one batch");
    const int s = *hs[i]->h_status;
    if (s != DLR_OK) return fail(s, "handle %d: %s", i, status_name(s));
  }
  return DLR_OK;
}

// the batch plan of a handle set (built on first use, then cached)
static int get_batch(dlr_handle *const *hs, int n, Batch **out) {
  int rc;
  if (n == 1) {
    if (!hs[0]->own_batch && (rc = build_batch(hs, 1, &hs[0]->own_batch))) return rc;
    *out = hs[0]->own_batch;
    return DLR_OK;
  }
  std::vector<dlr_handle *> key(hs, hs + n);
  auto &m = batch_cache();
  auto it = m.find(key);
  if (it == m.end()) {
    Batch *b = nullptr;
    if ((rc = build_batch(hs, n, &b))) return rc;
    m[key] = b;
    *out = b;
  } else {
    *out = it->second;
  }
  return DLR_OK;
}

int dlr_step_batch(dlr_handle *const *hs, int32_t n, int32_t nsteps) {
  int rc = check_handles(hs, n);
  if (rc) return rc;
  if (nsteps < 0) return fail(DLR_EINVAL, "nsteps < 0");
  if (nsteps == 0) return DLR_OK;
  Batch *b = nullptr;
  if ((rc = get_batch(hs, n, &b))) return rc;
  return run_steps(b, nsteps);
}

// Re-plans the batch's sweep units with splitting threshold `split`.
static int set_plan(Batch *b, double split) {
  std::vector<SiUnit> units;
  plan_units(b->hs.data(), b->n, b->mixed, b->grp, b->si_grid, split, units);
  if ((int)units.size() > b->units_cap) return fail(DLR_EINVAL, "unit plan exceeds its table");
  CK(cudaMemcpyAsync(b->d_units, units.data(), sizeof(SiUnit) * units.size(), cudaMemcpyHostToDevice,
                     b->st));
  b->ctl.n_units = (int)units.size();
  const int no_force = 0;  // timing runs of the autotuner leave a forced count behind
  CK(cudaMemcpyAsync(&b->gs->n_units, &b->ctl.n_units, sizeof(int), cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(&b->gs->force_iters, &no_force, sizeof(int), cudaMemcpyHostToDevice, b->st));
  CK(cudaStreamSynchronize(b->st));  // the host values die here
  b->split = split;
  return DLR_OK;
}

// Testing aid for the bounded waits: the finest plan, with the first unit
// that has an incoming edge row reading the spare row instead, which nothing
// writes.  The next step's wait for it gives up after its time bound and the
// instances report DLR_ETIMEOUT; nothing faults.
int dlr_debug_lose_edge(dlr_handle *const *hs, int32_t n) {
  int rc = check_handles(hs, n);
  if (rc) return rc;
  Batch *b = nullptr;
  if ((rc = get_batch(hs, n, &b))) return rc;
  std::vector<SiUnit> units;
  plan_units(b->hs.data(), b->n, b->mixed, b->grp, b->si_grid, 1e-9, units);
  auto it = std::find_if(units.begin(), units.end(), [](const SiUnit &u) { return u.in_row >= 0; });
  if (it == units.end()) return fail(DLR_EINVAL, "no angle spans more than one sweep unit");
  if ((int)units.size() > b->units_cap) return fail(DLR_EINVAL, "unit plan exceeds its table");
  it->in_row = b->spare_row;
  CK(cudaMemcpyAsync(b->d_units, units.data(), sizeof(SiUnit) * units.size(), cudaMemcpyHostToDevice,
                     b->st));
  b->ctl.n_units = (int)units.size();
  CK(cudaMemcpyAsync(&b->gs->n_units, &b->ctl.n_units, sizeof(int), cudaMemcpyHostToDevice, b->st));
  CK(cudaStreamSynchronize(b->st));
  return DLR_OK;
}

int dlr_set_split(dlr_handle *const *hs, int32_t n, double split) {
  int rc = check_handles(hs, n);
  if (rc) return rc;
  if (!(split >= 0) || split > 1e9) return fail(DLR_EINVAL, "split must be in [0, 1e9]");
  Batch *b = nullptr;
  if ((rc = get_batch(hs, n, &b))) return rc;
  return set_plan(b, split);
}

// The step's graphs of the batch (captured on first use, or after the
// source-iteration kernel was switched).
static int ensure_graphs(Batch *b) {
  int rc;
  if (!b->pre) {
    b->kcount = 0;
    if ((rc = capture(b, true, &b->pre))) return rc;
    if ((rc = capture(b, false, &b->post))) return rc;
    if (b->grp && (rc = capture_si(b))) return rc;
    b->kernels_per_step = b->kcount + 1;  // + source iteration (the last sweep of the grouped one)
  }
  return DLR_OK;
}

// Switches the batch between the grouped and the per-angle source-iteration
// kernel: the step's graphs are captured again (the coefficients go to the
// other kernel's layout) and the unit plan is redone for the kernel's items.
static int select_kernel(Batch *b, bool grp) {
  if (grp == b->grp) return DLR_OK;
  CK(cudaStreamSynchronize(b->st));
  for (cudaGraphExec_t *g : {&b->pre, &b->post, &b->si})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  b->grp = grp;
  b->si_grid = grp ? b->grid_grp : b->grid_angle;
  return set_plan(b, b->split);
}

// Times the source-iteration launch of the batch for each candidate sweep
// plan -- the splitting thresholds with the per-angle kernel, and again
// with the grouped kernel where the batch can take it (exactly `iters`
// iterations, `reps` launches after one untimed one) -- and keeps the
// fastest.  The sweeps run on the state the next step starts from (the
// "pre" graph of each kernel is replayed first); everything they write is
// recomputed by that step, and the iteration counters are left alone.
int dlr_autotune(dlr_handle *const *hs, int32_t n, int32_t iters, int32_t reps, double *chosen,
                 double *ms_out) {
  int rc = check_handles(hs, n);
  if (rc) return rc;
  if (iters < 1 || reps < 1) return fail(DLR_EINVAL, "iters and reps must be >= 1");
  Batch *b = nullptr;
  if ((rc = get_batch(hs, n, &b))) return rc;
  if ((rc = refresh_batch(b))) return rc;
  const double cand[] = {0.0, 2.0, 1.0, 0.5};
  const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
  auto same = [](const std::vector<SiUnit> &x, const std::vector<SiUnit> &y) {
    return x.size() == y.size() && std::memcmp(x.data(), y.data(), x.size() * sizeof(SiUnit)) == 0;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<double> ms(2 * nc, -1.0);  // per-angle kernel, then grouped
  int best = -1;
  cudaError_t e = cudaSuccess;
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    if (kind == 1 && !b->grp_ok) break;
    if ((rc = select_kernel(b, kind == 1)) || (rc = ensure_graphs(b))) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
    e = cudaGraphLaunch(b->pre, b->st);
    std::vector<std::vector<SiUnit>> plans(nc);
    for (int c = 0; c < nc; ++c) plan_units(b->hs.data(), n, b->mixed, b->grp, b->si_grid, cand[c], plans[c]);
    SiCtl c = b->ctl;
    c.force_iters = iters;
    for (int k = 0; k < nc && e == cudaSuccess; ++k) {
      const int slot = kind * nc + k;
      int dup = -1;
      for (int q = 0; q < k; ++q)
        if (same(plans[q], plans[k])) dup = q;
      if (dup >= 0) {
        ms[slot] = ms[kind * nc + dup];
        continue;
      }
      e = cudaMemcpyAsync(b->d_units, plans[k].data(), sizeof(SiUnit) * plans[k].size(),
                          cudaMemcpyHostToDevice, b->st);
      c.n_units = (int)plans[k].size();
      for (int rep = 0; rep <= reps && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, b->st);
        if (e == cudaSuccess)
          e = b->grp ? launch_grp_prep(b->d_insts, n, c, b->gs, b->st) : launch_si_prep(b->d_insts, n, c, b->st);
        if (e == cudaSuccess) e = launch_si_batch(b, c);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      ms[slot] = t / reps;
      if (best < 0 || ms[slot] < ms[best]) best = slot;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(DLR_ECUDA, "autotune: %s", cudaGetErrorString(e));
  const bool grp_best = best >= nc;
  b->split = cand[best % nc];
  if ((rc = select_kernel(b, grp_best))) return rc;
  if ((rc = set_plan(b, cand[best % nc]))) return rc;
  tune_table()[batch_shape(hs, n)] = TunedPlan{cand[best % nc], grp_best ? 1 : 0};
  for (auto *h : b->hs) {
    int s = 0;
    CK(cudaMemcpy(&s, h->inst.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (s != DLR_OK) {
      *h->h_status = s;
      return fail(s, "autotune: %s", status_name(s));
    }
  }
  if (chosen) *chosen = cand[best % nc];
  if (ms_out)
    for (int k = 0; k < 2 * nc; ++k) ms_out[k] = ms[k];
  return DLR_OK;
}

// ------------------------------------------------------------------
// getters / setters
// ------------------------------------------------------------------
static int sync_status(dlr_handle *h) {
  CK(cudaStreamSynchronize(h->st));
  int s = 0;
  CK(cudaMemcpy(&s, h->inst.status, sizeof(int), cudaMemcpyDeviceToHost));
  *h->h_status = s;
  if (s != DLR_OK) return fail(s, "%s", status_name(s));
  return DLR_OK;
}

int dlr_get_T(dlr_handle *h, double *out, int32_t out_on_device) {
  if (!h || !out) return fail(DLR_EINVAL, "NULL argument");
  CK(cudaMemcpyAsync(out, h->inst.T, (size_t)h->N * 8,
                     out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  return sync_status(h);
}

int dlr_set_T(dlr_handle *h, const double *in, int32_t in_on_device) {
  if (!h || !in) return fail(DLR_EINVAL, "NULL argument");
  CK(cudaMemcpyAsync(h->inst.T, in, (size_t)h->N * 8,
                     in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  return DLR_OK;
}

// Rotates the stored factors to the SVD basis of S (X0 <- X0 U, S0 <- Sigma,
// W0 <- W0 V, signs: largest-magnitude entry of each W column > 0); psi is
// unchanged.  Steps with pivoted-QR selection keep S general, because that
// selection depends only on span W.
static int canonicalize(dlr_handle *h) {
  if (h->canonical || h->aug) return DLR_OK;  // augmented factors are canonical after a step
  int rc;
  if (!h->own_batch && (rc = build_batch(&h, 1, &h->own_batch))) return rc;
  Batch *b = h->own_batch;
  rc = refresh_batch(b);
  if (rc) return rc;
  CK(launch_svd(b->d_insts, 1, 2, h->st));
  CK((launch_apply<double, double>(b->a_cw, 1, h->K, rank_mask(h->r), h->st)));
  CK(launch_sign(b->d_insts, 1, h->K, h->st));
  const int rowsX = h->inst.q1 ? 4 * h->N : h->N;  // rows of X0 (Q1: 4 per cell)
  if (h->mixed) CK((launch_apply<float, float>(b->a_cx, 1, rowsX, rank_mask(h->r), h->st)));
  else CK((launch_apply<double, double>(b->a_cx, 1, rowsX, rank_mask(h->r), h->st)));
  h->canonical = true;
  return DLR_OK;
}

// A rows x cols matrix of the working precision on the device, copied out
// to FP64 (host or device memory); with bilinear elements the stored rows
// are scaled and go out as plain Legendre coefficients.
static int copy_out(dlr_handle *h, const void *src, double *dst, size_t rows, int cols, bool on_device) {
  const size_t n = rows * cols;
  if (!h->mixed) {
    CK(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  } else if (on_device) {
    k_widen<<<1024, 256, 0, h->st>>>((const float *)src, dst, n);
    CK(cudaGetLastError());
  } else {
    std::vector<float> tmp(n);
    CK(cudaMemcpyAsync(tmp.data(), src, n * 4, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (size_t i = 0; i < n; ++i) dst[i] = tmp[i];
  }
  if (h->inst.q1) {
    if (on_device) {
      CK(launch_q1_rescale(dst, false, rows, cols, 1, h->st));
    } else {
      CK(cudaStreamSynchronize(h->st));
      for (size_t e = 0; e < n; ++e) dst[e] *= q1_unscale((int)((e % rows) & 3));
    }
  }
  return DLR_OK;
}

// The reverse of copy_out: FP64 (host or device) into the working precision.
static int copy_in(dlr_handle *h, void *dst, const double *src, size_t rows, int cols, bool on_device) {
  const size_t n = rows * cols;
  std::vector<double> scaled;
  if (h->inst.q1 && !on_device) {
    scaled.assign(src, src + n);
    for (size_t e = 0; e < n; ++e) scaled[e] *= q1_scale((int)((e % rows) & 3));
    src = scaled.data();
  }
  if (!h->mixed) {
    CK(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if (!on_device) CK(cudaStreamSynchronize(h->st));
  } else if (on_device) {
    k_narrow<<<1024, 256, 0, h->st>>>(src, (float *)dst, n);
    CK(cudaGetLastError());
  } else {
    std::vector<float> tmp(src, src + n);
    CK(cudaMemcpyAsync(dst, tmp.data(), n * 4, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  if (h->inst.q1 && on_device) CK(launch_q1_rescale(dst, h->mixed, rows, cols, 0, h->st));
  return DLR_OK;
}

int dlr_get_factors(dlr_handle *h, double *X, double *S, double *W, int32_t *r_out, int32_t out_on_device) {
  if (!h) return fail(DLR_EINVAL, "NULL handle");
  if (h->sn) return fail(DLR_EINVAL, "a full-rank SN handle has no factors (dlr_get_psi)");
  {
    int rc = canonicalize(h);
    if (rc) return rc;
  }
  const size_t rowsX = h->inst.q1 ? (size_t)4 * h->N : (size_t)h->N;
  const cudaMemcpyKind k = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (r_out) *r_out = h->r;
  if (X) {
    const int rc = copy_out(h, h->inst.X0, X, rowsX, h->r, out_on_device != 0);
    if (rc) return rc;
  }
  if (S) CK(cudaMemcpyAsync(S, h->inst.S0, (size_t)h->r * h->r * 8, k, h->st));
  if (W) CK(cudaMemcpyAsync(W, h->inst.W0, (size_t)h->K * h->r * 8, k, h->st));
  return sync_status(h);
}

int dlr_set_factors(dlr_handle *h, const double *X, const double *S, const double *W, int32_t in_on_device) {
  if (!h || !X || !S || !W) return fail(DLR_EINVAL, "NULL argument");
  if (h->sn) return fail(DLR_EINVAL, "a full-rank SN handle has no factors (dlr_set_psi)");
  h->canonical = false;
  const size_t rowsX = h->inst.q1 ? (size_t)4 * h->N : (size_t)h->N;
  const cudaMemcpyKind k = in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  {
    const int rc = copy_in(h, h->inst.X0, X, rowsX, h->r, in_on_device != 0);
    if (rc) return rc;
  }
  CK(cudaMemcpyAsync(h->inst.S0, S, (size_t)h->r * h->r * 8, k, h->st));
  CK(cudaMemcpyAsync(h->inst.W0, W, (size_t)h->K * h->r * 8, k, h->st));
  if (!in_on_device) CK(cudaStreamSynchronize(h->st));
  return DLR_OK;
}

int dlr_get_quadrature(dlr_handle *h, double *omega_xyz, double *w) {
  if (!h) return fail(DLR_EINVAL, "NULL handle");
  for (int k = 0; k < h->K; ++k) {
    if (omega_xyz) {
      omega_xyz[3 * k] = h->ox[k];
      omega_xyz[3 * k + 1] = h->oy[k];
      omega_xyz[3 * k + 2] = h->oz[k];
    }
    if (w) w[k] = h->w[k];
  }
  return DLR_OK;
}

int dlr_get_selected(dlr_handle *h, int32_t *idx) {
  if (!h || !idx) return fail(DLR_EINVAL, "NULL argument");
  if (h->sn) return fail(DLR_EINVAL, "a full-rank SN handle selects no angles");
  CK(cudaMemcpyAsync(idx, h->inst.idx, (size_t)h->r * 4, cudaMemcpyDeviceToHost, h->st));
  return sync_status(h);
}

int dlr_get_psi(dlr_handle *h, double *out, int32_t out_on_device) {
  if (!h || !out) return fail(DLR_EINVAL, "NULL argument");
  const size_t rows = h->inst.q1 ? (size_t)4 * h->N : (size_t)h->N;
  if (h->sn) {
    const int rc = copy_out(h, h->inst.Psi, out, rows, h->K, out_on_device != 0);
    if (rc) return rc;
    return sync_status(h);
  }
  // a DLR state: X S W^T formed on the device, into out or a scratch array,
  // from the factors in the SVD basis of S (as dlr_get_factors leaves them)
  {
    const int rc = canonicalize(h);
    if (rc) return rc;
  }
  const size_t bytes = rows * (size_t)h->K * 8;
  double *dst = out;
  if (!out_on_device) CK(cudaMallocAsync(reinterpret_cast<void **>(&dst), bytes, h->st));
  const dim3 g((unsigned)((rows + 127) / 128), (unsigned)h->K);
  if (h->mixed)
    k_form_psi<float><<<g, 128, 0, h->st>>>((const float *)h->inst.X0, rows, h->r, h->inst.S0, h->inst.W0, h->K,
                                             h->inst.q1, dst);
  else
    k_form_psi<double><<<g, 128, 0, h->st>>>((const double *)h->inst.X0, rows, h->r, h->inst.S0, h->inst.W0,
                                              h->K, h->inst.q1, dst);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !out_on_device) {
    e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->st);
    const cudaError_t f = cudaFreeAsync(dst, h->st);
    if (e == cudaSuccess) e = f;
  }
  if (e != cudaSuccess) return fail(DLR_ECUDA, "dlr_get_psi: %s", cudaGetErrorString(e));
  return sync_status(h);
}

int dlr_set_psi(dlr_handle *h, const double *in, int32_t in_on_device) {
  if (!h || !in) return fail(DLR_EINVAL, "NULL argument");
  if (!h->sn) return fail(DLR_EINVAL, "dlr_set_psi needs a full-rank SN handle (dlr_set_factors)");
  const size_t rows = h->inst.q1 ? (size_t)4 * h->N : (size_t)h->N;
  {
    const int rc = copy_in(h, h->inst.Psi, in, rows, h->K, in_on_device != 0);
    if (rc) return rc;
  }
  return DLR_OK;
}

int dlr_get_stats(dlr_handle *h, dlr_stats *out) {
  if (!h || !out) return fail(DLR_EINVAL, "NULL argument");
  CK(cudaStreamSynchronize(h->st));
  long long tot = 0;
  int last = 0, s = 0, np = 0;
  CK(cudaMemcpy(&np, h->inst.nonpos, sizeof np, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&tot, h->d_iters_total, sizeof tot, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&last, h->inst.iters, sizeof last, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&s, h->inst.status, sizeof s, cudaMemcpyDeviceToHost));
  for (auto &ev : h->ev_pending) {
    float a = 0, b2 = 0;
    cudaEventElapsedTime(&a, ev[1], ev[2]);
    cudaEventElapsedTime(&b2, ev[0], ev[3]);
    h->ms_si += a;
    h->ms_step += b2;
    h->si_launches += 1;
    for (auto e : ev) h->ev_pool.push_back(e);
  }
  h->ev_pending.clear();
  long long dsa_tot = 0;
  if (h->d_dsa_iters_total) CK(cudaMemcpy(&dsa_tot, h->d_dsa_iters_total, sizeof dsa_tot, cudaMemcpyDeviceToHost));
  out->dsa_iters_total = dsa_tot;
  out->steps = h->steps;
  out->si_iters_total = tot;
  out->cell_angle_updates = tot * (long long)h->N * h->r;
  out->si_iters_last = last;
  out->status = s;
  out->ms_si_total = h->ms_si;
  out->ms_step_total = h->ms_step;
  out->si_launches = h->si_launches;
  // the grouped source iteration launches three kernels per iteration
  out->kernel_launches = h->kernel_launches + (h->grp_loop ? 3 * tot : 0);
  out->sweep_grouped = h->grp_loop ? 1 : 0;
  out->nonpositive_cells = np;
  int rp = 0;
  if (h->inst.refl_passes) CK(cudaMemcpy(&rp, h->inst.refl_passes, sizeof rp, cudaMemcpyDeviceToHost));
  out->refl_passes_last = rp;
  *h->h_status = s;
  return DLR_OK;
}

int dlr_set_timing(dlr_handle *h, int32_t enable) {
  if (!h) return fail(DLR_EINVAL, "NULL handle");
  h->timing = enable != 0;
  return DLR_OK;
}

int dlr_set_edge_inflow(dlr_handle *h, int32_t edge, double psi_iso) {
  if (!h || edge < 0 || edge > 3 || !(psi_iso >= 0) || !std::isfinite(psi_iso))
    return fail(DLR_EINVAL, "bad edge or inflow value");
  h->inst.psi_edge[edge] = psi_iso;
  ++h->version;
  return DLR_OK;
}

namespace dlr {
// The standalone sweep keeps a band's top row in shared memory, so the mesh
// width is bounded by the device's opt-in shared memory per block: DLR_OK,
// or DLR_EINVAL (with its message) for a mesh too wide.  Checked before any
// work is enqueued, so a refused call leaves no runtime error behind.
int sweep_width_check(int nx, int ny, int precision) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(DLR_ECUDA, "no usable current device");
  }
  const int bands = (ny + 31) / 32;
  const size_t need = precision == DLR_MIXED ? si_smem_bytes<float>(nx, bands, 0, 0, 0)
                                             : si_smem_bytes<double>(nx, bands, 0, 0, 0);
  if (optin > 0 && need > (size_t)optin)
    return fail(DLR_EINVAL, "nx = %d too large for the sweep's shared memory", nx);
  return DLR_OK;
}
}  // namespace dlr

int dlr_sweep(int32_t nx, int32_t ny, double lx, double ly, int32_t n_dir, const double *dirs,
              const double *psi_edge, int32_t precision, const void *sigma_t, const void *src,
              void *psi, void *stream) {
  if (nx < 1 || ny < 1 || n_dir < 1 || !dirs || !psi_edge || !sigma_t || !src || !psi || !(lx > 0) ||
      !(ly > 0) || (precision != DLR_FP64 && precision != DLR_MIXED))
    return fail(DLR_EINVAL, "bad argument to dlr_sweep");
  if (int rc = sweep_width_check(nx, ny, precision)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double *d_dirs = nullptr, *d_edge = nullptr;
  int *d_abort = nullptr;
  CK(cudaMallocAsync(&d_dirs, (size_t)n_dir * 2 * 8, st));
  CK(cudaMallocAsync(&d_edge, 4 * 8, st));
  CK(cudaMallocAsync(&d_abort, sizeof(int), st));
  CK(cudaMemcpyAsync(d_dirs, dirs, (size_t)n_dir * 2 * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_edge, psi_edge, 4 * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d_abort, 0, sizeof(int), st));
  const double hx = lx / nx, hy = ly / ny;
  cudaError_t e = precision == DLR_MIXED
                      ? launch_sweep_dirs<float>(nx, ny, hx, hy, n_dir, d_dirs, d_edge, (const float *)sigma_t,
                                                 (const float *)src, (float *)psi, d_abort, st)
                      : launch_sweep_dirs<double>(nx, ny, hx, hy, n_dir, d_dirs, d_edge,
                                                  (const double *)sigma_t, (const double *)src, (double *)psi,
                                                  d_abort, st);
  if (e != cudaSuccess) return fail(DLR_ECUDA, "sweep launch failed: %s", cudaGetErrorString(e));
  int ab = 0;
  CK(cudaMemcpyAsync(&ab, d_abort, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaFreeAsync(d_dirs, st));
  CK(cudaFreeAsync(d_edge, st));
  CK(cudaFreeAsync(d_abort, st));
  CK(cudaStreamSynchronize(st));
  if (ab) return fail(DLR_ETIMEOUT, "a sweep wait timed out");
  return DLR_OK;
}
