// dlr_internal.cuh -- device-side data layout and helpers shared by the
// kernels of the SN-like DLR step (Algorithm 1 of Haut et al.).
//
// Layout of one instance in HBM (r = rank, N = nx*ny cells, K = angles):
//   real  X0[N*r], X[N*r], Psi[N*r], s0[N*r]   column-major (cell fastest)
//   real  sig_t[N], ss4[N] (= sigma_s / 4pi), q[N], phi[2][N], sphi[N]
//   f64   T[N], B0[N], D[N], sigma[N], rho_cv[N]
//   f64   W0[K*r] (column-major), S0[r*r], L[r*K] (angle-major rows of r)
//   f64   small[]   r x r work matrices (offsets in SmallLayout)
//   f64   lu[K*r*r], int piv[K*r]  per-angle LU factors of B_k
//   f64   partials[] per-cluster partial sums of the tall-skinny reductions
// "real" is float in mixed precision and double in FP64 mode.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dlr {

namespace cg = cooperative_groups;

constexpr int kMaxRank = 32;
// CTAs per thread-block cluster of the tall-skinny reductions: the CTAs of a
// cluster sum their partials through distributed shared memory, so one
// partial per cluster reaches global memory.
constexpr int kCl = 8;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTieRel = 1e-12;  // angle-selection tie window

// status codes mirror include/dlr.h
constexpr int kOk = 0;
constexpr int kENotConv = -3;
constexpr int kESingular = -4;
constexpr int kETimeout = -5;
constexpr int kENonPos = -6;

// Offsets (in doubles) of the r x r work matrices inside Inst::small.
struct SmallLayout {
  int What, Winv, beta, gamma, C0;     // angle selection
  int R1, R2, R3;                      // CholeskyQR factors
  int qr_flag;    // ints: [0] third pass needed, [1] filled columns, [2..] mask
  int G, Nx, Ny, Mt, Ms, P, vec;       // projections (vec: qh, bL, bR, bB, bT)
  int Axp, Axm, Ayp, Aym, PS0;         // L-step operators
  int Cbar, zeta, Lbar, tvec;          // C-bar device
  int RGx, RGy, RHx, RHy;              // reflective edges (DLR)
  int U, V, sv, vphi, Sn, Tr;          // SVD of S and temperature vector
  int total;
};

inline SmallLayout small_layout(int r) {
  SmallLayout s;
  int o = 0;
  auto m = [&](int n) { int at = o; o += n; return at; };
  s.What = m(r * r); s.Winv = m(r * r); s.beta = m(r); s.gamma = m(r); s.C0 = m(r * r);
  s.R1 = m(r * r); s.R2 = m(r * r); s.R3 = m(r * r); s.qr_flag = m(20);
  s.G = m(r * r); s.Nx = m(r * r); s.Ny = m(r * r); s.Mt = m(r * r); s.Ms = m(r * r);
  s.P = m(r * r); s.vec = m(5 * r);
  s.Axp = m(r * r); s.Axm = m(r * r); s.Ayp = m(r * r); s.Aym = m(r * r); s.PS0 = m(r * r);
  s.Cbar = m(r * r); s.zeta = m(r); s.Lbar = m(r); s.tvec = m(r);
  s.RGx = m(r * r); s.RGy = m(r * r); s.RHx = m(r * r); s.RHy = m(r * r);
  s.U = m(r * r); s.V = m(r * r); s.sv = m(r); s.vphi = m(r); s.Sn = m(r * r); s.Tr = m(r * r);
  s.total = o;
  return s;
}

// Thresholds of the CholeskyQR passes (chol_core.cuh).  u: a pivot below
// u tr(G) needs a shift.  tau: in the first pass, a column whose residual^2
// is below tau |column|^2 is dependent and replaced by an orthonormal
// completion.  The Gram resolves a residual^2 only to a few ulps of
// |column|^2, so in FP64 tau sits above that level (1e-14, about 45 ulps: a
// column within about 1e-7 of the span of the previous ones, e.g. the
// collocation fluxes of an exactly isotropic state, counts as dependent).  In
// mixed precision the FP32 Grams resolve only about 1e-6, which would also
// catch genuine columns at rank 32; tau stays at 1e-10 there.
__host__ __device__ inline double chol_u(bool mixed) { return mixed ? 1e-7 : 1e-15; }
__host__ __device__ inline double chol_tau(bool mixed) { return mixed ? 1e-10 : 1e-14; }

// Number of doubles one block writes for each reduction kind.
// (six r x r matrices G, Nx, Ny, Mt, Ms, P and five r-vectors per block)
__host__ __device__ inline int proj_count(int r) { return 6 * r * r + 5 * r; }

struct Inst {
  int nx, ny, N, r, K;
  int precision, selection, fixed_iters, max_iter;
  double hx, hy, h2, dt, c, a_rad, inv_cdt, si_tol;
  double psi_edge[4];
  // per cell, FP64
  const double *sigma, *rho_cv;
  double *T, *B0, *D;
  // per cell, real
  void *sig_t, *ss4, *q, *phi0, *phi1, *sphi;
  // N x r, real
  void *X0, *X, *Psi, *s0;
  // quadrature, FP64
  const double *ox, *oy, *w;
  // factors, FP64
  double *W0, *S0, *L;
  double *Lf;              // L with dependent rows replaced (QR input)
  // angle selection
  int *idx;
  // r x r work space and per-angle LU
  double *small;
  SmallLayout lay;
  double *lu;
  int *piv;
  // partial sums of block reductions (partial_stride doubles per block)
  double *partials;
  int partial_blocks;      // CTAs of the cell reductions (project, Gram; whole clusters)
  int angle_blocks;        // CTAs of the angle reductions (Grams of L; whole clusters)
  int lstep_blocks;        // blocks of the per-angle L-step
  // status and iteration bookkeeping
  int *status;            // sticky device status
  int *nonpos;            // cells with T <= 0 after the last step
  int allow_nonpos;       // 1: count non-positive T instead of failing
  int *iters;             // iterations of the last source-iteration solve
  unsigned long long *iters_total;  // iterations summed over all steps
  unsigned long long *conv;  // [2 parities][2]: max |dphi|, max |phi| (bits)
  // full-rank SN instances: r = K swept angles, idx the identity, and the
  // scalar-flux weights gamma = w read from here (nullptr: the DLR gamma in
  // small)
  int method;
  const double *gamma_ext;
  // augmented step (rank-2r basis truncated back to rank r): in the rank-r
  // instance aug_x0 is where step 3 copies X0 (the second half of the
  // [Psi, X0] input of step 5); in the rank-2r instance aug_r = r and S0_r is
  // the rank-r S0 that the truncation writes
  int aug_r;
  void *aug_x0;
  double *S0_r;
  // temperature-dependent materials, taken at the step's T0:
  // sigma(T) = sigma (T/T_ref)^-sig_texp, rho c_v(T) = rho_cv (T/T_ref)^cv_texp
  double sig_texp, cv_texp, T_ref;
  // diffusion synthetic acceleration of the source iteration (Section 4.5;
  // dsa = 0: off).  Per cell (real): 1/sigma_t, the diagonal of the DSA
  // operator and its inverse, and the CG vectors.  dsa_cx = 1/(12 hx^2),
  // dsa_kx = kappa_x / hx (likewise in y): the stencil scaled by 1/h^2.
  int dsa, dsa_max_iter;
  double dsa_tol, dsa_cx, dsa_cy, dsa_kx, dsa_ky;
  void *dsa_ist, *dsa_dg, *dsa_dinv, *dsa_x, *dsa_r, *dsa_z, *dsa_p0, *dsa_p1, *dsa_q;
  unsigned long long *dsa_iters_total;  // CG iterations summed over all steps
  // reflective edges (full-rank SN; left, right, bottom, top): a direction
  // entering a reflective edge takes, row by row, its mirror direction's
  // boundary value from the previous source iteration.  The sweep sees that
  // inflow as a source: the scalar inflow of the edge is 0 and the upwind
  // term (|Om_x|/hx) psi_in is added to the angle's fixed source s0 in the
  // boundary cells.  refl_base (real, K x (ny + nx), nullptr without
  // reflective edges) keeps those cells' own fixed source: entry
  // k (ny + nx) + o for boundary row o (o < ny) of the x-edge angle k enters,
  // and for boundary column o - ny of its y-edge
  int reflect[4];
  int n_azim;
  // 1: the angles of polar cosines +-mu (polar indices p and n_polar - 1 - p)
  // have bitwise equal Om_x, Om_y, so step 7 forms B_k^{-1} once per pair
  int polar_pairs;
  void *refl_base;
  // reflective edges of a DLR instance (reading R19; refl_base then holds
  // r x (ny + nx) entries, one per chosen angle j).  In the source iteration
  // the inflow of chosen angle j through a reflective edge is its mirror
  // angle's value interpolated through the chosen angles, G Psi(c) with
  // G = W0(Om_R(idx)) What^{-1} (small: RGx, RGy; RHx, RHy = C0 G^T give it
  // from X0 in the first sweeps).  Step 7 solves its reflected inflow by a
  // fixed point on the boundary values: refl_kap (FP64, (2 ny + 2 nx) x r)
  // What^{-1} Psi(c) of the boundary cells (left, right, bottom, top),
  // refl_data (FP64, K x (ny + nx)) the boundary value of each (angle,
  // entry), refl_y and refl_u (FP64, K x r) B_k^{-1} Q_k and B_k^{-1}
  // g_k, refl_passes the fixed-point passes of the last step.
  double *refl_kap, *refl_data, *refl_y, *refl_u;
  int *refl_passes;
  // bilinear (Q1) elements (k_q1.cu): X0, X, Psi, s0 are 4 N x r, phi0,
  // phi1 4 N (real), rows e = 4 c + m scaled by (1, 1/sqrt3, 1/sqrt3, 1/3);
  // q1_wt, q1_ws (FP64, 4 N) the row weights sigma_t, sigma_s of the step-7
  // mass Grams, q1_v (real, 4 N x r) the transport operator applied to X
  int q1;
  double *q1_wt, *q1_ws;
  void *q1_v;
  // grouped-angle sweep (mixed-precision DLR instances without DSA or
  // reflective edges, grp = 1): the chosen angles are grouped by quadrant
  // (kGA per group, table grp_tab of grp_ng records, ordered by quadrant),
  // and the sweep's inputs and outputs live in the skewed band layout of
  // grp_off (glay floats per layout, glay / 1024 blocks): sgk holds per
  // group and block the kGA angles' fixed sources and sigma_t of the
  // group's quadrant, (kGA + 1) x 1024 floats together (grp_sgk); spk
  // sigma_s phi / 4 pi in the four quadrant layouts, two sets for the
  // iteration parity; part per group the sum over its angles of
  // gamma_j psi_j; qsum per quadrant the sum of its groups' part
  int grp, grp_ng, nwin, nbands;
  size_t glay;
  int *grp_tab;
  float *sgk, *spk, *part, *qsum;
};

// Bilinear (Q1) coefficients are stored scaled by s = (1, 1/sqrt3, 1/sqrt3,
// 1/3) (k_q1.cu): q1_scale(m) = s_m, q1_unscale(m) = 1/s_m.
constexpr double kQ1Sqrt3 = 1.7320508075688772935;
__host__ __device__ inline double q1_scale(int m) { return m == 0 ? 1.0 : (m == 3 ? 1.0 / 3.0 : 1.0 / kQ1Sqrt3); }
__host__ __device__ inline double q1_unscale(int m) { return m == 0 ? 1.0 : (m == 3 ? 3.0 : kQ1Sqrt3); }

// Angles per group of the grouped sweep, and the ints of one group record:
// quadrant, number of angles, the angles' indices j.
constexpr int kGA = 2;
constexpr int kGrpRec = 2 + kGA;
// Groups needed for r angles in any split over the four quadrants.
__host__ __device__ inline int grp_count(int r) { return (r + 4 * (kGA - 1)) / kGA; }

// Skewed band layout of the grouped sweep.  Quadrant quad = (Om_x < 0) +
// 2 (Om_y < 0) mirrors the mesh so that its directions point to +u, +v
// (u = x or nx-1-x, v = y or ny-1-y).  Rows are grouped in bands of 32
// (lane i = v mod 32 of band b = v / 32); lane i reaches column u at
// wavefront step t = u + i, and step t belongs to window k = t / 32.  One
// (band, window) block holds 32 lanes x 32 steps, lane-major (a lane's 32
// steps in one 128-byte row), the 4-step groups of a row permuted by
// XOR with i mod 8 so that the lanes' 16-byte reads of one step group fall
// in distinct banks.  Blocks are 4 KB and ordered (band, window); nwin =
// (nx + 62) / 32 windows cover t = 0 .. nx + 30.  Positions outside the
// mesh are padding.
__host__ __device__ inline int grp_nwin(int nx) { return (nx + 62) >> 5; }
__host__ __device__ inline size_t grp_lay(int nx, int ny) {
  return (size_t)((ny + 31) >> 5) * grp_nwin(nx) * 1024;
}
__device__ __forceinline__ size_t grp_off(int quad, int nx, int ny, int nwin, int x, int y) {
  const int u = (quad & 1) ? nx - 1 - x : x;
  const int v = (quad & 2) ? ny - 1 - y : y;
  const int i = v & 31, t = u + i;
  const int s = t & 31;
  return ((size_t)((v >> 5) * nwin + (t >> 5)) << 10) + (i << 5) + ((((s >> 2) ^ (i & 7)) << 2) | (s & 3));
}
__device__ __forceinline__ int quad_of(double ox, double oy) { return (ox < 0 ? 1 : 0) | (oy < 0 ? 2 : 0); }
// Position in sgk of slot `slot` (0 .. kGA-1: the group's angles, kGA:
// sigma_t) of group g at layout offset o (block o / 1024, entry o % 1024).
__host__ __device__ inline size_t grp_sgk(size_t glay, int g, int slot, size_t o) {
  return ((((size_t)g * (glay >> 10) + (o >> 10)) * (kGA + 1) + slot) << 10) + (o & 1023);
}

// Mirror image of quadrature angle k = p n_azim + a of the product
// quadrature: axis 0 negates the x component (azimuth a -> n_azim/2 - 1 - a,
// n_azim even), axis 1 the y component (a -> n_azim - 1 - a).
__host__ __device__ inline int mirror_angle(int k, int n_azim, int axis) {
  const int p = k / n_azim, a = k - p * n_azim;
  const int b = axis == 0 ? (n_azim / 2 - 1 - a + n_azim) % n_azim : n_azim - 1 - a;
  return p * n_azim + b;
}

__device__ __forceinline__ double sigma_at(const Inst &I, int c, double T0) {
  return I.sig_texp == 0.0 ? I.sigma[c] : I.sigma[c] * pow(T0 / I.T_ref, -I.sig_texp);
}
__device__ __forceinline__ double rhocv_at(const Inst &I, int c, double T0) {
  return I.cv_texp == 0.0 ? I.rho_cv[c] : I.rho_cv[c] * pow(T0 / I.T_ref, I.cv_texp);
}

// Rank classes of the kernels unrolled over RB = 8, 16 or 32 columns: a
// batch launches one kernel per class present, each skipping the other
// instances, so an instance's work follows its own rank.
__host__ __device__ inline int rank_class(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : 32; }
__host__ __device__ inline int rank_mask(int r) { return r <= 8 ? 1 : r <= 16 ? 2 : 4; }

// Per-cell coefficients of the Newton-linearised step (Section 2.2, in the
// backward-Euler form: D = rho c_v + 4 pi dt sigma B'(T0), effective
// scattering sigma_s = sigma 4 pi dt sigma B' / D, effective source
// q = sigma B0 - sigma B' 4 pi dt sigma B0 / D, with B = a c T^4 / (4 pi)).
struct CellCoef {
  double B, D, ss, q, sig;  // sig = sigma(T0)
};
__device__ __forceinline__ CellCoef cell_coefficients(const Inst &I, int c) {
  const double T0 = I.T[c], sig = sigma_at(I, c, T0), rho = rhocv_at(I, c, T0);
  CellCoef k;
  k.sig = sig;
  k.B = I.a_rad * I.c * T0 * T0 * T0 * T0 / (4.0 * kPi);
  const double dB = I.a_rad * I.c * T0 * T0 * T0 / kPi;
  const double g = 4.0 * kPi * I.dt * sig * dB;
  k.D = rho + g;
  k.ss = sig * g / k.D;
  k.q = sig * k.B - sig * dB * (4.0 * kPi * I.dt * sig * k.B) / k.D;
  return k;
}

// Work descriptors of the batched kernels (one entry per instance).
// A tall-skinny Gram: m x r matrix A, layout 0 column-major A[row + lda*i],
// layout 1 rows of r contiguous A[i + r*row]; optional row weights.
struct GramJob {
  const void *A;
  const double *wt;
  int m, r, lda, layout;
  const void *B;    // optional: cross Gram sum wt a b^T with B (layout 0, ldb)
  int ldb;
  int sqrt_wt;      // 1: weight sqrt(wt) instead of wt
  double *out;      // partial sums, one r x r block per cluster
  int nblocks;      // CTAs used for this job (a multiple of kCl)
  const int *run_if;  // optional: skip unless *run_if != 0
};

// out = diag(s_out) (diag(s_in) A) T for a small r x r T (FP64); with tri
// set, T holds an upper-triangular R and out = diag(s_out) (diag(s_in) A) R^-1
// (forward substitution per row).
struct ApplyJob {
  const void *A;        // input (real_in)
  int in_layout;        // 0: column-major (lda), 1: rows of r contiguous
  int lda;
  const double *s_in;   // optional per-row scale (sqrt applied if sq_in)
  int sq_in;
  const double *T;      // r x r column-major FP64
  void *out;            // column-major, leading dimension ldo
  int ldo;
  const double *s_out;  // optional per-row scale
  int inv_sq_out;       // 1: multiply by 1/sqrt(s_out)
  int m, r;
  int tri;              // 1: T is upper triangular, apply its inverse
  const int *run_if;  // optional: skip unless *run_if != 0
};

struct ReduceJob {
  const double *part;
  int nblocks, stride, count;
  double *out;
  double scale;
};

struct CholJob {
  const double *part;
  int nblocks;      // partials (clusters) to sum
  double scale;
  double *R;        // upper-triangular factor (applied by forward substitution)
  int *flag;        // ints: [0] third pass needed, [1] filled columns, [2..] mask
  int r;
  int mode;         // 1 detect, 2 plain, 3 only if flag[0], 4 only if flag[1]
  double u;         // relative size of the shift (data precision)
  double tau_dep;   // a column whose residual^2 falls below tau_dep |col|^2 is dependent
};

// Copies a tall-skinny matrix (optionally) and replaces the columns marked
// dependent by deterministic pseudo-random ones (orthonormal completion).
struct FillJob {
  void *A;          // matrix to fill (layout as in GramJob)
  const void *src;  // if non-null: copy src into A first (same layout)
  int m, r, lda, layout;
  const int *flag;  // CholJob flag block
};

// One unit of sweep work: bands b0 .. b0 + nb - 1 (32 rows each) of one
// angle of one instance.  An angle whose bands are split over several units
// hands the top row of each unit's last band to the next unit through a row
// of a global edge table (in_row / out_row, -1 if none).
struct SiUnit {
  int inst, angle, b0, nb, in_row, out_row;
};

struct SiCtl {
  unsigned *bar;        // [0] arrivals, [1] generation
  unsigned *work;       // [2] unit counters by iteration parity
  int *abort_flag;
  const SiUnit *units;  // in claiming order: a unit's predecessor comes first
  int n_units;
  int n_inst;
  int nx_max, bands_max;
  int gam_max;                 // largest r of the batch (scalar-flux weights in shared memory)
  unsigned long long *gedge;   // edge rows between units: n_rows x gedge_ld words, each
                               // column one (FP32) or two (FP64) words tag << 32 | bits
  unsigned *epoch;             // launch counter (tags of the edge words)
  int n_rows, gedge_ld;
  int force_iters;             // > 0: every instance runs exactly this many iterations
                               // and its iteration counters are left alone (timing runs)
  int any_dsa;                 // some instance accelerates its iteration (Section 4.5)
  double *dsa_part;            // per-CTA partial sums of the DSA CG: n_inst x kDsaSlots x grid
};

// Loop state of the grouped source iteration (one per batch, device
// memory): the iteration index, the blocks of the scalar-flux kernel that
// have finished, a forced iteration count (timing runs), the number of
// sweep units, and per instance whether it is still iterating and the
// parity of its last sweep's sigma_s phi (-1: not swept in this step).
struct GrpSi {
  int it;
  unsigned done;
  int force_iters;
  int n_units;
  int *active;
  int *par_of;
  double *relax;  // relaxation state per instance (3 each, see relax_track)
};

// partial sums of one DSA CG iteration: p.q, r.z, r.r, and b.b of the
// right-hand side
constexpr int kDsaSlots = 4;
// per-cell device arrays of the DSA solve
constexpr int kDsaArrays = 9;

// Four consecutive elements, aligned for one vector shared-memory access.
template <typename real> struct alignas(4 * sizeof(real)) Quad { real v[4]; };

template <typename real> struct Real2;
template <> struct Real2<float> { using type = float2; };
template <> struct Real2<double> { using type = double2; };

// fused multiply-add in the precision of the arguments (a plain fma() call
// with float arguments would be evaluated in FP64)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Deterministic pseudo-random value in [-1, 1) from a 64-bit key (the
// SplitMix64 finaliser); used for the orthonormal completion of dependent
// columns.
__device__ __forceinline__ double hash_uniform(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <typename T>
__device__ __forceinline__ T *as(void *p) { return reinterpret_cast<T *>(p); }
template <typename T>
__device__ __forceinline__ const T *as_c(const void *p) { return reinterpret_cast<const T *>(p); }

// Programmatic dependent launch (launch_pdl): a kernel may be scheduled while
// its predecessor in the stream (or graph) is still running, which hides the
// launch gap between the many short kernels of a step.  Every such kernel
// calls pdl_wait() before it reads anything a predecessor writes, and
// pdl_trigger() to let its own successor be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// First error wins; later ones are dropped.
__device__ __forceinline__ void set_status(int *status, int code) {
  atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Non-negative doubles order like their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// sum_b part[b * stride + e] for b < nb with eight independent partial sums
// (loads in flight together; the order of the additions is fixed, so the
// result is deterministic).
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int nb,
                                               size_t stride, size_t e) {
  double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int b = 0;
  for (; b + 8 <= nb; b += 8) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] += part[(size_t)(b + q) * stride + e];
  }
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (b + q < nb) a[q] += part[(size_t)(b + q) * stride + e];
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// Block-wide sum; every thread gets the result.  scratch >= 32 entries.
template <typename T>
__device__ T block_sum(T v, T *scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T t = lane < nw ? scratch[lane] : T(0);
  t = warp_sum(t);
  return t;
}
template <typename T>
__device__ T block_max(T v, T *scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T t = lane < nw ? scratch[lane] : T(-1e308);
  t = warp_max(t);
  return t;
}

// The boundary-cell geometry of angle k: the x-edge and y-edge it enters
// (0 left, 1 right, 2 bottom, 3 top), the boundary column and row, and the
// upwind coefficients |Om_x|/hx, |Om_y|/hy in the working precision.
template <typename real>
struct ReflGeom {
  int ex, ey, bx, by;
  bool rx, ry;
  real ax, ay;
  __device__ __forceinline__ ReflGeom(const Inst &I, int k) {
    ex = I.ox[k] > 0 ? 0 : 1;
    ey = I.oy[k] > 0 ? 2 : 3;
    bx = ex == 0 ? 0 : I.nx - 1;
    by = ey == 2 ? 0 : I.ny - 1;
    rx = I.reflect[ex] != 0;
    ry = I.reflect[ey] != 0;
    ax = real(fabs(I.ox[k]) / I.hx);
    ay = real(fabs(I.oy[k]) / I.hy);
  }
};

// The reflected inflow of swept angle j (quadrature angle k) in boundary
// cell c through its x-edge (axis 0) or y-edge (axis 1), from the sweeps'
// output psi (N x r): full-rank SN takes the mirror direction's own value
// (reading R18); DLR interpolates the mirror angle through the chosen ones,
// sum_m G_jm Psi(c, m) with G = RGx or RGy (reading R19).
template <typename real>
__device__ __forceinline__ real refl_in(const Inst &I, const real *psi, int j, int k, int c, int axis) {
  if (!I.refl_kap) return psi[(size_t)I.N * mirror_angle(k, I.n_azim, axis) + c];
  const double *G = I.small + (axis == 0 ? I.lay.RGx : I.lay.RGy);
  real v = real(0);
  for (int m = 0; m < I.r; ++m) v = fmadd(real(G[j + I.r * m]), psi[(size_t)I.N * m + c], v);
  return v;
}

// Entry e of refl_base (see Inst): the fixed source of its boundary cell
// plus the reflected inflow term(s) from psi (N x r) of the swept angles,
// written to s0.  The corner cell of two reflective edges is written by its
// x-edge entry only.
template <typename real>
__device__ __forceinline__ void refl_inject(const Inst &I, const real *psi, int e) {
  const int L = I.ny + I.nx, j = e / L, o = e - j * L;
  const int k = I.refl_kap ? I.idx[j] : j;
  const ReflGeom<real> G(I, k);
  const real *base = as_c<real>(I.refl_base) + (size_t)j * L;
  real *s0 = as<real>(I.s0) + (size_t)I.N * j;
  if (o < I.ny) {
    if (!G.rx) return;
    const int c = o * I.nx + G.bx;
    real v = fmadd(G.ax, refl_in<real>(I, psi, j, k, c, 0), base[o]);
    if (G.ry && o == G.by) v = fmadd(G.ay, refl_in<real>(I, psi, j, k, c, 1), v);
    s0[c] = v;
  } else {
    const int ix = o - I.ny;
    if (!G.ry || (G.rx && ix == G.bx)) return;
    const int c = G.by * I.nx + ix;
    s0[c] = fmadd(G.ay, refl_in<real>(I, psi, j, k, c, 1), base[o]);
  }
}

// Relaxation of the collocation source iteration (reading R22): the update
// phi <- phi + omega (phi^{l+1/2} - phi) starts with omega = 1 (the plain
// iteration); each time the sweeps' change d = max|phi^{l+1/2} - phi| has
// grown by more than kRelaxGrow for kRelaxRun consecutive iterations while
// above kRelaxMin max|phi^{l+1/2}|, omega is halved (a diverging iteration
// whose dominant eigenvalue is below -1 becomes a contraction), down to
// kRelaxFloor; a further such run means the relaxed iteration diverges too
// (returns true: the step ends with DLR_ENOTCONV).  The omega of an update
// is the one decided after the previous iteration; the state per instance
// is (omega, the previous d, the growth run).
constexpr double kRelaxGrow = 1.05, kRelaxMin = 1e-4, kRelaxFloor = 0.125;
constexpr int kRelaxRun = 3;
__host__ __device__ inline bool relax_track(double d, double m, double *st) {
  bool give_up = false;
  if (st[1] >= 0.0 && d > kRelaxGrow * st[1] && d > kRelaxMin * m) {
    st[2] += 1.0;
    if (st[2] >= kRelaxRun) {
      if (st[0] <= kRelaxFloor) give_up = true;
      st[0] *= 0.5;
      st[2] = 0.0;
    }
  } else {
    st[2] = 0.0;
  }
  st[1] = d;
  return give_up;
}
__host__ __device__ inline void relax_reset(double *st) {
  st[0] = 1.0;
  st[1] = -1.0;
  st[2] = 0.0;
}

constexpr uint64_t kGridWaitNs = 4000000000ull;  // bound of a grid-barrier wait

// Sense-reversing grid barrier with a bounded wait (co-residency of all
// CTAs is guaranteed by the cooperative launch).  A wait that runs out sets
// the abort flag, so that every CTA leaves at its next wait and the launch
// reports the timeout.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, volatile int *abort_flag) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint64_t t0 = global_ns();
      unsigned spins = 0;
      while (*gen == g) {
        if ((++spins & 63u) == 0) {
          __nanosleep(64);
          if (*abort_flag) { ok = 0; break; }
          if (global_ns() - t0 > kGridWaitNs) {
            *abort_flag = 1;
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    ok_s = ok && !*abort_flag;
  }
  __syncthreads();
  return ok_s;
}

}  // namespace dlr
