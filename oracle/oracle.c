/*
 * oracle.c -- plain, slow, FP64 CPU reference of the SN-like DLR time step
 * (Haut et al., Section 4, Algorithm 1) on a 2-D Cartesian mesh with a DG0
 * (piecewise-constant, upwind "step") spatial discretisation.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product library.  It shares no
 * code with the CUDA path.  Every function cites the passage it follows.
 * Readings of the paper used here (where it is silent or garbled):
 *   R1  Newton-linearised coefficients derived from Eq. (T, backward Euler):
 *       D = rho_cv + 4 pi dt sigma B'(T0),  T = T0 + dt sigma (phi - 4 pi B0)/D,
 *       sigma_s = sigma (4 pi dt sigma B')/D,  q = sigma B0 rho_cv / D.
 *       (The printed q and T-update carry an extra rho_cv T0 term that breaks
 *       equilibrium; the derivation is redone from the backward-Euler form.)
 *   R2  B(T) = a c T^4/(4 pi)  (gray Planck), so B' = a c T^3 / pi.
 *   R4  isotropic inflow psi_edge on an edge for directions entering it.
 *   R5  product quadrature: Gauss-Legendre in mu x equispaced azimuths.
 *   R6  DG0 upwind cells: the lowest-order member of the paper's upwind DG.
 *   R7  SI stops when max|phi_new - phi| <= tol * max|phi_new|.
 *   R8  angle choice: column-pivoted Householder QR of W^T (default) or the
 *       greedy DEIM of Section 4.2; ties go to the lowest index within a
 *       relative 1e-12 of the maximum.
 *   R10 What_ij = W_j(Om^(i)); Psi = What K; phi = beta^T What^{-1} Psi.
 *   R11 initial factors: psi0(x, Om) = B(T0(x)), S0 = diag(s0, 0, ...).
 *   R12 the temperature update uses phi of the final factors, X S beta.
 *   R15 augmented step (optional; Algorithm 1 never forms rank 2r): the
 *       rank-2r rounding the paper gives for its PN-like method (Section 3)
 *       carried over to the SN-like step -- the new basis is
 *       orth([Psi, X0]) (2r columns, h^2 inner product), steps 6-8 run at
 *       rank 2r (P = <X^, X0> is 2r x r), and the 2r x 2r S = U Sigma V^T is
 *       truncated to its r largest singular values (X = X^ U_r, S = Sigma_r,
 *       W = W V_r, signs as in the canonical form) before step 9.
 *   R16 temperature-dependent materials (no law is given): per-cell power
 *       laws sigma(T) = sigma (T/T_ref)^-n_s, rho c_v(T) = rho_cv (T/T_ref)^n_c,
 *       taken at the step's T0 as Eq. (T, backward Euler) prescribes (the
 *       transport opacity too: sigma_t = sigma(T0) + 1/(c dt)).
 *   R17 DSA (Section 4.5) on DG0 cells: the volume terms G_j vanish on
 *       piecewise constants, faces on the domain boundary see a zero
 *       exterior trace (the vacuum error equation), and the penalty F0 uses
 *       the full-quadrature coefficient (1/4 pi)(1/2) sum_k w_k |Om_k . n|,
 *       the traditional consistent-DSA penalty the paper's experiments use,
 *       in place of the collocation weights beta^T What^{-1}.  The DSA
 *       system A delta = M_s (phi^{l+1/2} - phi^l) is solved by
 *       Jacobi-preconditioned CG to ||r||_2 <= dsa_tol ||b||_2 (at most
 *       dsa_max_iter iterations), and phi^{l+1} = phi^{l+1/2} + delta.
 *       The stopping test of R7 is applied to the sweep's change,
 *       phi^{l+1/2} - phi^l (what it measures without DSA): the
 *       correction multiplies rounding noise by up to sigma_s / sigma_a in
 *       thick scattering cells, so phi^{l+1} - phi^l would stall above a
 *       tolerance near the working precision.
 *   R18 reflective edges (full-rank SN): a direction entering through a
 *       reflective edge takes as inflow, row by row, the boundary cell value
 *       of its mirror image (the direction with the normal component
 *       negated), from the previous source iteration (from psi^n in the
 *       first); the product quadrature maps onto itself (x mirror: azimuth
 *       a -> n_azim/2 - 1 - a, needs n_azim even; y mirror: a -> n_azim - 1
 *       - a).
 *   R20 DSA on Q1 elements: the DG derivative is
 *       v^T D_j u = -sum_K int_K u dv/dx_j + sum_faces int {u} [[v]]_j
 *       (the volume term G_j of Section 4.4 with the face term in the form
 *       that makes D_j exact for continuous fields, which on piecewise
 *       constants is the centred difference of R17), M_t and M_a the Q1
 *       mass matrices weighted by sigma_t and sigma_a, F0 the face-jump
 *       penalty of R17 on the Q1 traces, zero traces outside.
 *   R19 reflective edges in the DLR step: the collocation sweeps take the
 *       mirror direction's boundary value interpolated through the chosen
 *       angles (W0(Om_R)^T What^-1 Psi) from the previous source
 *       iteration; the L-step's reflected inflow X(c) L_R(k) is implicit and
 *       solved by a fixed point on the boundary values (per-angle L-steps
 *       with the current values as extra inflow).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads: where OpenMP is available, loops whose iterations are independent
 * (angles of one round of sweeps, cells of the scalar flux, columns of a
 * reflector application, entries of a projection, angles of the L-step)
 * run in parallel.  Every sum keeps its serial order inside one iteration
 * and no iteration writes what another reads, so the results are bitwise
 * those of one thread. */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}
int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

#define ORACLE_PI 3.14159265358979323846
#define TIE_REL 1e-12

/* ------------------------------------------------------------------ */
/* Physics: Section 2.1 (Eq. TRT psi, TRT T) and Section 2.2.          */
/* ------------------------------------------------------------------ */

double oracle_planck(double a_rad, double c, double T) {
  return a_rad * c * T * T * T * T / (4.0 * ORACLE_PI);
}

/* dB/dT of the gray Planck function (reading R2). */
static double planck_deriv(double a_rad, double c, double T) {
  return a_rad * c * T * T * T / ORACLE_PI;
}

/* sigma(T0) and rho c_v(T0) of cell c (Section 2.1, taken explicitly at
 * T0 as in Eq. T backward Euler; reading R16 for the law). */
static double tref(const oracle_problem *p) { return p->T_ref > 0 ? p->T_ref : 1.0; }
double oracle_sigma_at(const oracle_problem *p, int c, double T0) {
  if (p->sigma_texp == 0.0) return p->sigma[c];
  return p->sigma[c] * pow(T0 / tref(p), -p->sigma_texp);
}
double oracle_rhocv_at(const oracle_problem *p, int c, double T0) {
  if (p->cv_texp == 0.0) return p->rho_cv[c];
  return p->rho_cv[c] * pow(T0 / tref(p), p->cv_texp);
}

/* Section 2.2: Newton linearisation of the backward-Euler temperature
 * equation about T0 gives the pseudo-scattering sigma_s (Eq. effective
 * scattering) and the source q (Eq. effective source; reading R1). */
void oracle_coefficients(const oracle_problem *p, const double *T0,
                         double *sigma_s, double *q, double *B0, double *D) {
  int Nx = p->nx * p->ny;
  for (int c = 0; c < Nx; c++) {
    double sig = oracle_sigma_at(p, c, T0[c]);
    double B = oracle_planck(p->a_rad, p->c, T0[c]);
    double dB = planck_deriv(p->a_rad, p->c, T0[c]);
    double Dc = oracle_rhocv_at(p, c, T0[c]) + 4.0 * ORACLE_PI * p->dt * sig * dB;
    sigma_s[c] = sig * (4.0 * ORACLE_PI * p->dt * sig * dB) / Dc;
    q[c] = sig * B - sig * dB * (4.0 * ORACLE_PI * p->dt * sig * B) / Dc;
    if (B0) B0[c] = B;
    if (D) D[c] = Dc;
  }
}

/* ------------------------------------------------------------------ */
/* Quadrature (reading R5).                                            */
/* ------------------------------------------------------------------ */

/* Legendre P_n and its derivative at z by the three-term recurrence. */
static void legendre(int n, double z, double *Pn, double *dPn) {
  double p0 = 1.0, p1 = z;
  if (n == 0) { *Pn = 1.0; *dPn = 0.0; return; }
  for (int k = 2; k <= n; k++) {
    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *Pn = p1;
  *dPn = n * (z * p1 - p0) / (z * z - 1.0);
}

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1]: roots of P_n by
 * Newton's method, weights 2 / ((1 - z^2) P_n'(z)^2). */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; i++) {
    double z = cos(ORACLE_PI * (i + 0.75) / (n + 0.5));
    double Pn, dPn;
    for (int it = 0; it < 200; it++) {
      legendre(n, z, &Pn, &dPn);
      double dz = Pn / dPn;
      z -= dz;
      if (fabs(dz) < 1e-15) {
        legendre(n, z, &Pn, &dPn);
        z -= Pn / dPn;
        break;
      }
    }
    legendre(n, z, &Pn, &dPn);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dPn * dPn);
  }
}

void oracle_quadrature(int n_polar, int n_azim, double *ox, double *oy,
                       double *oz, double *w) {
  double *mu = (double *)malloc(sizeof(double) * n_polar);
  double *wp = (double *)malloc(sizeof(double) * n_polar);
  gauss_legendre(n_polar, mu, wp);
  for (int p = 0; p < n_polar; p++) {
    double s = sqrt(1.0 - mu[p] * mu[p]);
    for (int a = 0; a < n_azim; a++) {
      double phi = (a + 0.5) * 2.0 * ORACLE_PI / n_azim;
      int k = p * n_azim + a;
      ox[k] = s * cos(phi);
      oy[k] = s * sin(phi);
      oz[k] = mu[p];
      w[k] = wp[p] * 2.0 * ORACLE_PI / n_azim;
    }
  }
  free(mu);
  free(wp);
}

/* ------------------------------------------------------------------ */
/* DG0 upwind transport sweep (Section 4.4 discretisation, reading R6). */
/* ------------------------------------------------------------------ */

/* Inflow value entering through the x-face of the first cell of a row for
 * direction sign ox, and through the y-face for oy (reading R4). */
static double inflow_x(const oracle_problem *p, double ox) {
  return ox > 0 ? p->psi_edge[0] : (ox < 0 ? p->psi_edge[1] : 0.0);
}
static double inflow_y(const oracle_problem *p, double oy) {
  return oy > 0 ? p->psi_edge[2] : (oy < 0 ? p->psi_edge[3] : 0.0);
}

/* Cell balance of the upwind scheme: integrating Om.grad psi over cell c and
 * taking the upwind face values gives
 *   |ox|/hx (psi_c - psi_west) + |oy|/hy (psi_c - psi_south)
 *       + sigma_t,c psi_c = src_c,
 * where west/south are the upwind neighbours (or the edge inflow).  The
 * sweep solves this lower-triangular system cell by cell in upwind order. */
void oracle_sweep_in(const oracle_problem *p, double ox, double oy,
                     const double *sigma_t, const double *src,
                     const double *in_x, const double *in_y, double *psi) {
  int nx = p->nx, ny = p->ny;
  double hx = p->lx / nx, hy = p->ly / ny;
  double ax = fabs(ox) / hx, ay = fabs(oy) / hy;
  int sx = ox >= 0 ? 1 : -1, sy = oy >= 0 ? 1 : -1;
  for (int jj = 0; jj < ny; jj++) {
    int iy = sy > 0 ? jj : ny - 1 - jj;
    for (int ii = 0; ii < nx; ii++) {
      int ix = sx > 0 ? ii : nx - 1 - ii;
      int c = iy * nx + ix;
      double up_x = ii == 0 ? in_x[iy] : psi[iy * nx + (ix - sx)];
      double up_y = jj == 0 ? in_y[ix] : psi[(iy - sy) * nx + ix];
      psi[c] = (src[c] + ax * up_x + ay * up_y) / (sigma_t[c] + ax + ay);
    }
  }
}

void oracle_sweep(const oracle_problem *p, double ox, double oy,
                  const double *sigma_t, const double *src, double *psi) {
  double *in_x = (double *)malloc(sizeof(double) * p->ny);
  double *in_y = (double *)malloc(sizeof(double) * p->nx);
  for (int iy = 0; iy < p->ny; iy++) in_x[iy] = inflow_x(p, ox);
  for (int ix = 0; ix < p->nx; ix++) in_y[ix] = inflow_y(p, oy);
  oracle_sweep_in(p, ox, oy, sigma_t, src, in_x, in_y, psi);
  free(in_x); free(in_y);
}

/* Reflection maps of the product quadrature (reading R18). */
int oracle_reflect_index(int n_polar, int n_azim, int k, int axis) {
  int pp = k / n_azim, a = k % n_azim;
  int b = axis == 0 ? ((n_azim / 2 - 1 - a) % n_azim + n_azim) % n_azim : n_azim - 1 - a;
  (void)n_polar;
  return pp * n_azim + b;
}

/* Inflow of every angle through the edges it enters (reading R4; R18 on
 * reflective edges, from psi, Nx x NOm): in_x[k ny + iy], in_y[k nx + ix]. */
static void sn_inflow(const oracle_problem *p, const double *ox, const double *oy,
                      const double *psi, double *in_x, double *in_y) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim;
  for (int k = 0; k < NOm; k++) {
    int ex = ox[k] > 0 ? 0 : 1, ey = oy[k] > 0 ? 2 : 3;
    int kx = oracle_reflect_index(p->n_polar, p->n_azim, k, 0);
    int ky = oracle_reflect_index(p->n_polar, p->n_azim, k, 1);
    for (int iy = 0; iy < ny; iy++) {
      int c = iy * nx + (ex == 0 ? 0 : nx - 1);
      in_x[k * ny + iy] = p->reflect[ex] ? psi[c + (size_t)Nx * kx] : inflow_x(p, ox[k]);
    }
    for (int ix = 0; ix < nx; ix++) {
      int c = (ey == 2 ? 0 : ny - 1) * nx + ix;
      in_y[k * nx + ix] = p->reflect[ey] ? psi[c + (size_t)Nx * ky] : inflow_y(p, oy[k]);
    }
  }
}

/* ------------------------------------------------------------------ */
/* Bilinear (Q1) upwind DG sweep (Section 4.4 with bilinear elements). */
/* ------------------------------------------------------------------ */

/* On cell [xc - a, xc + a] x [yc - b, yc + b] (a = hx/2, b = hy/2) a Q1
 * function is u = u0 + u1 xi + u2 eta + u3 xi eta in the reference
 * coordinates xi = (x - xc)/a, eta = (y - yc)/b.  The cell equations are
 * the upwind DG weak form of Section 4.4 (the volume term of G_j and the
 * face matrix F_d): for every basis function v,
 *   -int_K u (Om . grad v) + sum_faces int (Om . n) u^ v + int_K sigma_t u v
 *       = int_K src v,
 * with u^ the own trace on outflow faces and the upwind trace (the
 * neighbour's, or the inflow) on inflow faces.  The inflow on a boundary
 * face is a linear function along it: in[0] + in[1] s, s in [-1, 1] the
 * reference coordinate along the face (eta on x-faces, xi on y-faces).
 * src and psi hold 4 coefficients per cell (cell-major); in_x[2 iy + m]
 * is the inflow of row iy through the upwind x-face, in_y[2 ix + m] that
 * of column ix through the upwind y-face. */

static int lu_factor(int n, double *A, int *piv);
static void lu_solve_inplace(int n, const double *LU, const int *piv, double *b);
static int lstep_solve(const oracle_problem *p, int r, double *const *Ax, double *const *Ay,
                       const double *Mt, const double *Ms, const double *qh,
                       double *const *bE, const double *Lt0, const double *gext, double *L);
static double *dsa_matrix_q1_new(const oracle_problem *p, const double *sig_t, const double *sig_s);
static int dsa_correct_q1(const oracle_problem *p, const double *A, const double *sig_s,
                          const double *phi_old, double *phi_half);
static int relax_track(double dmax, double pmax, double *dprev, int *grow, double *omega);

/* int_{-1}^{1} of the products of two face traces, each trace written as
 * (c + d s) with (c, d) = (t0, t1): the face trace of basis function i is
 * tr[i][0] + tr[i][1] s. */
static double face_prod(const double *ti, const double *tj) {
  return 2.0 * ti[0] * tj[0] + (2.0 / 3.0) * ti[1] * tj[1];
}

/* Face traces (constant, slope along the face) of 1, xi, eta, xi eta:
 * x-faces xi = +-1 (slope in eta), y-faces eta = +-1 (slope in xi). */
static const double Q1_TR_R[4][2] = {{1, 0}, {1, 0}, {0, 1}, {0, 1}};
static const double Q1_TR_L[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
static const double Q1_TR_T[4][2] = {{1, 0}, {0, 1}, {1, 0}, {0, 1}};
static const double Q1_TR_B[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
static const double Q1_MASS[4] = {4.0, 4.0 / 3.0, 4.0 / 3.0, 4.0 / 9.0};

/* The transport part of the cell matrix (volume term and outflow faces) of
 * direction (ox, oy) on a cell of half-widths a, b: A[i + 4 j]. */
static void q1_local(double ox, double oy, double a, double b, double *A) {
  const double (*tout_x)[2] = ox >= 0 ? Q1_TR_R : Q1_TR_L;
  const double (*tout_y)[2] = oy >= 0 ? Q1_TR_T : Q1_TR_B;
  for (int e = 0; e < 16; e++) A[e] = 0.0;
  /* volume: -int u (Om . grad v) = -(ox b D1 + oy a D2), with
   * int int (d v_i / d xi) v_j: (1,0) -> 4, (3,2) -> 4/3 and
   * int int (d v_i / d eta) v_j: (2,0) -> 4, (3,1) -> 4/3 */
  A[1 + 4 * 0] -= ox * b * 4.0;
  A[3 + 4 * 2] -= ox * b * 4.0 / 3.0;
  A[2 + 4 * 0] -= oy * a * 4.0;
  A[3 + 4 * 1] -= oy * a * 4.0 / 3.0;
  /* outflow faces: |Om . n| (face length / 2) int trace_i trace_j */
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++)
      A[i + 4 * j] += fabs(ox) * b * face_prod(tout_x[i], tout_x[j]) +
                      fabs(oy) * a * face_prod(tout_y[i], tout_y[j]);
}

/* The trace, on the shared face, of the upwind neighbour's coefficients un
 * (axis 0: the neighbour across the x-face the direction enters, s = sign
 * of ox; axis 1 likewise in y), as (constant, slope). */
static void q1_upwind_trace(const double *un, int axis, int s, double *tr) {
  const double (*tn)[2] = axis == 0 ? (s > 0 ? Q1_TR_R : Q1_TR_L) : (s > 0 ? Q1_TR_T : Q1_TR_B);
  tr[0] = tr[1] = 0.0;
  for (int j = 0; j < 4; j++) {
    tr[0] += un[j] * tn[j][0];
    tr[1] += un[j] * tn[j][1];
  }
}

/* The inflow-face terms |Om . n| (length / 2) int u^ trace_i of the traces
 * ux, uy entering through the upwind x- and y-faces, added to r. */
static void q1_inflow_terms(double ox, double oy, double a, double b, const double *ux,
                            const double *uy, double *r) {
  const double (*tin_x)[2] = ox >= 0 ? Q1_TR_L : Q1_TR_R;
  const double (*tin_y)[2] = oy >= 0 ? Q1_TR_B : Q1_TR_T;
  for (int i = 0; i < 4; i++)
    r[i] += fabs(ox) * b * face_prod(tin_x[i], ux) + fabs(oy) * a * face_prod(tin_y[i], uy);
}

void oracle_sweep_q1(const oracle_problem *p, double ox, double oy,
                     const double *sigma_t, const double *src,
                     const double *in_x, const double *in_y, double *psi) {
  int nx = p->nx, ny = p->ny;
  double hx = p->lx / nx, hy = p->ly / ny, a = 0.5 * hx, b = 0.5 * hy;
  int sx = ox >= 0 ? 1 : -1, sy = oy >= 0 ? 1 : -1;
  double A[16], rhs[4], ux[2], uy[2];
  int piv[4];
  for (int jj = 0; jj < ny; jj++) {
    int iy = sy > 0 ? jj : ny - 1 - jj;
    for (int ii = 0; ii < nx; ii++) {
      int ix = sx > 0 ? ii : nx - 1 - ii;
      int c = iy * nx + ix;
      q1_local(ox, oy, a, b, A);
      /* reaction and source (the Legendre mass matrix is diagonal) */
      for (int i = 0; i < 4; i++) {
        A[i + 4 * i] += sigma_t[c] * a * b * Q1_MASS[i];
        rhs[i] = a * b * Q1_MASS[i] * src[4 * c + i];
      }
      if (ii == 0) {
        ux[0] = in_x[2 * iy];
        ux[1] = in_x[2 * iy + 1];
      } else {
        q1_upwind_trace(psi + 4 * (iy * nx + ix - sx), 0, sx, ux);
      }
      if (jj == 0) {
        uy[0] = in_y[2 * ix];
        uy[1] = in_y[2 * ix + 1];
      } else {
        q1_upwind_trace(psi + 4 * ((iy - sy) * nx + ix), 1, sy, uy);
      }
      q1_inflow_terms(ox, oy, a, b, ux, uy, rhs);
      if (lu_factor(4, A, piv) != 0) {
        for (int i = 0; i < 4; i++) psi[4 * c + i] = NAN;
        continue;
      }
      lu_solve_inplace(4, A, piv, rhs);
      memcpy(psi + 4 * c, rhs, sizeof rhs);
    }
  }
}

/* The transport operator of direction (ox, oy) on Q1 fields, without
 * sigma and with zero boundary inflow: out = the left-hand side of the cell
 * equations of the sweep (tested against every basis function) for u. */
static void q1_transport_apply(const oracle_problem *p, double ox, double oy, const double *u,
                               double *out) {
  int nx = p->nx, ny = p->ny;
  double a = 0.5 * p->lx / nx, b = 0.5 * p->ly / ny;
  int sx = ox >= 0 ? 1 : -1, sy = oy >= 0 ? 1 : -1;
  double A[16], ux[2], uy[2], inr[4];
  q1_local(ox, oy, a, b, A);
  for (int iy = 0; iy < ny; iy++)
    for (int ix = 0; ix < nx; ix++) {
      int c = iy * nx + ix;
      for (int i = 0; i < 4; i++) {
        double t = 0;
        for (int j = 0; j < 4; j++) t += A[i + 4 * j] * u[4 * c + j];
        out[4 * c + i] = t;
      }
      int jx = ix - sx, jy = iy - sy;
      ux[0] = ux[1] = uy[0] = uy[1] = 0.0;
      if (jx >= 0 && jx < nx) q1_upwind_trace(u + 4 * (iy * nx + jx), 0, sx, ux);
      if (jy >= 0 && jy < ny) q1_upwind_trace(u + 4 * (jy * nx + ix), 1, sy, uy);
      for (int i = 0; i < 4; i++) inr[i] = 0.0;
      q1_inflow_terms(ox, oy, a, b, ux, uy, inr);
      for (int i = 0; i < 4; i++) out[4 * c + i] -= inr[i];
    }
}

/* Full-rank SN step on Q1 elements (Section 2.2 with the sweep above):
 * psi holds 4 Legendre coefficients per cell for every angle,
 * psi[4 (k Nx + c) + m]; the materials and T stay per cell (the emission q
 * is constant on a cell), and the temperature update takes the cell
 * average of phi (its constant coefficient).  Returns the source
 * iterations, or -2 at the cap. */
int oracle_sn_step_q1(const oracle_problem *p, double *psi, double *T,
                      double si_tol, int si_max_iter, double *phi_out,
                      double *outflow, double *inflow) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim;
  double hx = p->lx / nx, hy = p->ly / ny, inv_cdt = 1.0 / (p->c * p->dt);
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  double *sig_s = (double *)malloc(sizeof(double) * Nx);
  double *q = (double *)malloc(sizeof(double) * Nx);
  double *B0 = (double *)malloc(sizeof(double) * Nx);
  double *D = (double *)malloc(sizeof(double) * Nx);
  double *sig_t = (double *)malloc(sizeof(double) * Nx);
  double *phi = (double *)calloc(4 * (size_t)Nx, sizeof(double));
  double *phin = (double *)malloc(sizeof(double) * 4 * Nx);
  double *src = (double *)malloc(sizeof(double) * 4 * Nx);
  double *psi0 = (double *)malloc(sizeof(double) * 4 * (size_t)Nx * NOm);
  double *in_x = (double *)malloc(sizeof(double) * 2 * ny);
  double *in_y = (double *)malloc(sizeof(double) * 2 * nx);
  memcpy(psi0, psi, sizeof(double) * 4 * (size_t)Nx * NOm);
  oracle_coefficients(p, T, sig_s, q, B0, D);
  for (int c = 0; c < Nx; c++) sig_t[c] = oracle_sigma_at(p, c, T[c]) + inv_cdt;
  for (int k = 0; k < NOm; k++)
    for (size_t e = 0; e < 4 * (size_t)Nx; e++) phi[e] += w[k] * psi0[4 * (size_t)Nx * k + e];
  int iters = 0, converged = 0;
  double *Adsa = p->dsa ? dsa_matrix_q1_new(p, sig_t, sig_s) : NULL;
  while (iters < si_max_iter) {
    for (size_t e = 0; e < 4 * (size_t)Nx; e++) phin[e] = 0;
    for (int k = 0; k < NOm; k++) {
      for (int c = 0; c < Nx; c++)
        for (int m = 0; m < 4; m++)
          src[4 * c + m] = sig_s[c] * phi[4 * c + m] / (4.0 * ORACLE_PI) + (m == 0 ? q[c] : 0.0) +
                           inv_cdt * psi0[4 * ((size_t)Nx * k + c) + m];
      for (int iy = 0; iy < ny; iy++) { in_x[2 * iy] = inflow_x(p, ox[k]); in_x[2 * iy + 1] = 0; }
      for (int ix = 0; ix < nx; ix++) { in_y[2 * ix] = inflow_y(p, oy[k]); in_y[2 * ix + 1] = 0; }
      double *pk = psi + 4 * (size_t)Nx * k;
      oracle_sweep_q1(p, ox[k], oy[k], sig_t, src, in_x, in_y, pk);
      for (size_t e = 0; e < 4 * (size_t)Nx; e++) phin[e] += w[k] * pk[e];
    }
    iters++;
    double dmax = 0, pmax = 0;
    int bad = 0;  /* a non-finite scalar flux: the iteration diverged */
    for (size_t e = 0; e < 4 * (size_t)Nx; e++) {
      if (!isfinite(phin[e])) bad = 1;
      if (fabs(phin[e] - phi[e]) > dmax) dmax = fabs(phin[e] - phi[e]);
      if (fabs(phin[e]) > pmax) pmax = fabs(phin[e]);
    }
    if (bad) break;
    if (p->dsa) dsa_correct_q1(p, Adsa, sig_s, phi, phin);  /* R17, R20 */
    memcpy(phi, phin, sizeof(double) * 4 * Nx);
    if (dmax <= si_tol * pmax) { converged = 1; break; }
  }
  for (int c = 0; c < Nx; c++)
    T[c] = T[c] + p->dt * oracle_sigma_at(p, c, T[c]) * (phi[4 * c] - 4.0 * ORACLE_PI * B0[c]) / D[c];
  if (phi_out) memcpy(phi_out, phi, sizeof(double) * 4 * Nx);
  if (outflow && inflow) {
    /* face means of the traces: right u0 + u1, left u0 - u1, top u0 + u2,
     * bottom u0 - u2 */
    double o = 0, i_ = 0;
    for (int k = 0; k < NOm; k++) {
      const double *pk = psi + 4 * (size_t)Nx * k;
      for (int iy = 0; iy < ny; iy++) {
        const double *u = pk + 4 * (iy * nx + (ox[k] < 0 ? 0 : nx - 1));
        o += w[k] * fabs(ox[k]) * hy * (u[0] + (ox[k] < 0 ? -u[1] : u[1]));
        i_ += w[k] * fabs(ox[k]) * hy * inflow_x(p, ox[k]);
      }
      for (int ix = 0; ix < nx; ix++) {
        const double *u = pk + 4 * ((oy[k] < 0 ? 0 : ny - 1) * nx + ix);
        o += w[k] * fabs(oy[k]) * hx * (u[0] + (oy[k] < 0 ? -u[2] : u[2]));
        i_ += w[k] * fabs(oy[k]) * hx * inflow_y(p, oy[k]);
      }
    }
    *outflow = o;
    *inflow = i_;
  }
  free(ox); free(oy); free(oz); free(w); free(sig_s); free(q); free(B0); free(D);
  free(sig_t); free(phi); free(phin); free(src); free(psi0); free(in_x); free(in_y); free(Adsa);
  return converged ? iters : -2;
}

/* One SN-like DLR step (Algorithm 1) on Q1 elements, steps 2-9 in the
 * order of Algorithm 1 with the Q1 sweep in step 4 and the Q1 transport
 * operator in step 7.  X (4 Nx x r) holds Q1 coefficients, orthonormal in
 * the L2 inner product of Q1 fields, int_K u v = sum_m wq_m u_m v_m with
 * wq = hx hy (1, 1/3, 1/3, 1/9); S, W as for DG0; T per cell (its update
 * takes the cell average of phi).  Angle choice by pivoted QR; no
 * canonical rotation of the factors; DSA (R17, R20) when p->dsa.  Returns 0, -1 (bad input, singular
 * matrix) or -2 (SI cap); iters_out and phi_out (4 Nx) may be NULL. */
int oracle_dlr_step_q1(const oracle_problem *p, int r, double *X, double *S, double *W,
                       double *T, double si_tol, int si_max_iter, int *iters_out,
                       double *phi_out) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, M4 = 4 * Nx, NOm = p->n_polar * p->n_azim;
  double hx = p->lx / nx, hy = p->ly / ny, inv_cdt = 1.0 / (p->c * p->dt);
  if (r < 1 || r > M4 || r > NOm) return -1;
  int rc = 0;
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  double *wq = (double *)malloc(sizeof(double) * M4);
  for (int c = 0; c < Nx; c++)
    for (int m = 0; m < 4; m++) wq[4 * c + m] = hx * hy * Q1_MASS[m] / 4.0;

  /* step 1: coefficients from T0 */
  double *sig_s = (double *)malloc(sizeof(double) * Nx);
  double *q = (double *)malloc(sizeof(double) * Nx);
  double *B0 = (double *)malloc(sizeof(double) * Nx);
  double *D = (double *)malloc(sizeof(double) * Nx);
  double *sig_t = (double *)malloc(sizeof(double) * Nx);
  oracle_coefficients(p, T, sig_s, q, B0, D);
  for (int c = 0; c < Nx; c++) sig_t[c] = oracle_sigma_at(p, c, T[c]) + inv_cdt;

  /* step 2: angles, What, beta */
  int *idx = (int *)calloc(r, sizeof(int)); /* valid indices even if the choice fails */
  double *WLU = (double *)malloc(sizeof(double) * r * r);
  int *wpiv = (int *)malloc(sizeof(int) * r);
  double *beta = (double *)calloc(r, sizeof(double));
  if (oracle_qdeim(NOm, r, W, idx) != 0) rc = -1;
  for (int i = 0; i < r; i++)
    for (int j = 0; j < r; j++) WLU[i + r * j] = W[idx[i] + (size_t)NOm * j];
  for (int j = 0; j < r; j++)
    for (int k = 0; k < NOm; k++) beta[j] += w[k] * W[k + (size_t)NOm * j];
  if (rc == 0 && lu_factor(r, WLU, wpiv) != 0) rc = -1;

  /* step 3: psi0 at the chosen angles, Psi0_j = X L0[:, idx_j], L0 = S W^T */
  double *L0 = (double *)malloc(sizeof(double) * r * NOm);
  for (int i = 0; i < r; i++)
    for (int k = 0; k < NOm; k++) {
      double t = 0;
      for (int l = 0; l < r; l++) t += S[i + r * l] * W[k + (size_t)NOm * l];
      L0[i + r * k] = t;
    }
  double *Psi0 = (double *)malloc(sizeof(double) * M4 * r);
  double *Psi = (double *)malloc(sizeof(double) * M4 * r);
  for (int j = 0; j < r; j++)
    for (int e = 0; e < M4; e++) {
      double t = 0;
      for (int i = 0; i < r; i++) t += X[e + (size_t)M4 * i] * L0[i + r * idx[j]];
      Psi0[e + (size_t)M4 * j] = t;
    }

  /* step 4: source iteration; phi = beta^T What^-1 Psi per coefficient */
  double *phi = (double *)malloc(sizeof(double) * M4);
  double *phin = (double *)malloc(sizeof(double) * M4);
  double *src = (double *)malloc(sizeof(double) * M4);
  double *Kc = (double *)malloc(sizeof(double) * r);
  double *in_x = (double *)malloc(sizeof(double) * 2 * ny);
  double *in_y = (double *)malloc(sizeof(double) * 2 * nx);
  int iters = 0;
  double *Adsa = p->dsa ? dsa_matrix_q1_new(p, sig_t, sig_s) : NULL;
  if (rc == 0) {
    for (int e = 0; e < M4; e++) {
      for (int j = 0; j < r; j++) Kc[j] = Psi0[e + (size_t)M4 * j];
      lu_solve_inplace(r, WLU, wpiv, Kc);
      double t = 0;
      for (int j = 0; j < r; j++) t += beta[j] * Kc[j];
      phi[e] = t;
    }
    int converged = 0;
    double omega = 1.0, dprev = -1.0;  /* relaxation state (reading R22) */
    int grow = 0;
    while (iters < si_max_iter) {
      for (int j = 0; j < r; j++) {
        int k = idx[j];
        for (int c = 0; c < Nx; c++)
          for (int m = 0; m < 4; m++)
            src[4 * c + m] = sig_s[c] * phi[4 * c + m] / (4.0 * ORACLE_PI) + (m == 0 ? q[c] : 0.0) +
                             inv_cdt * Psi0[4 * c + m + (size_t)M4 * j];
        for (int iy = 0; iy < ny; iy++) { in_x[2 * iy] = inflow_x(p, ox[k]); in_x[2 * iy + 1] = 0; }
        for (int ix = 0; ix < nx; ix++) { in_y[2 * ix] = inflow_y(p, oy[k]); in_y[2 * ix + 1] = 0; }
        oracle_sweep_q1(p, ox[k], oy[k], sig_t, src, in_x, in_y, Psi + (size_t)M4 * j);
      }
      iters++;
      double dmax = 0, pmax = 0;
      int bad = 0;  /* a non-finite scalar flux: the iteration diverged */
      for (int e = 0; e < M4; e++) {
        for (int j = 0; j < r; j++) Kc[j] = Psi[e + (size_t)M4 * j];
        lu_solve_inplace(r, WLU, wpiv, Kc);
        double t = 0;
        for (int j = 0; j < r; j++) t += beta[j] * Kc[j];
        phin[e] = t;
        if (!isfinite(t)) bad = 1;
        if (fabs(t - phi[e]) > dmax) dmax = fabs(t - phi[e]);
        if (fabs(t) > pmax) pmax = fabs(t);
      }
      if (bad) break;
      if (p->dsa) {
        dsa_correct_q1(p, Adsa, sig_s, phi, phin);  /* R17, R20 */
        memcpy(phi, phin, sizeof(double) * M4);
      } else {
        if (omega == 1.0) memcpy(phi, phin, sizeof(double) * M4);
        else
          for (int e = 0; e < M4; e++) phi[e] += omega * (phin[e] - phi[e]);
        if (relax_track(dmax, pmax, &dprev, &grow, &omega)) break;
      }
      if (dmax <= si_tol * pmax) { converged = 1; break; }
    }
    if (!converged) rc = -2;
  }
  if (iters_out) *iters_out = iters;

  /* step 5: Psi = X R, X orthonormal in the Q1 inner product */
  double *Xn = (double *)malloc(sizeof(double) * M4 * r);
  double *R = (double *)malloc(sizeof(double) * r * r);
  double *A = (double *)malloc(sizeof(double) * M4 * r);
  if (rc == 0) {
    for (int j = 0; j < r; j++)
      for (int e = 0; e < M4; e++) A[e + (size_t)M4 * j] = sqrt(wq[e]) * Psi[e + (size_t)M4 * j];
    oracle_householder_qr(M4, r, A, Xn, R);
    for (int j = 0; j < r; j++)
      for (int e = 0; e < M4; e++) Xn[e + (size_t)M4 * j] /= sqrt(wq[e]);
  }

  /* step 6: Lt0 = P L0, P = <X_new, X_old> */
  double *Lt0 = (double *)malloc(sizeof(double) * r * NOm);
  double *P = (double *)malloc(sizeof(double) * r * r);
  if (rc == 0) {
    for (int jj = 0; jj < r; jj++)
      for (int i = 0; i < r; i++) {
        double t = 0;
        for (int e = 0; e < M4; e++) t += Xn[e + (size_t)M4 * jj] * wq[e] * X[e + (size_t)M4 * i];
        P[jj + r * i] = t;
      }
    for (int jj = 0; jj < r; jj++)
      for (int k = 0; k < NOm; k++) {
        double t = 0;
        for (int i = 0; i < r; i++) t += P[jj + r * i] * L0[i + r * k];
        Lt0[jj + r * k] = t;
      }
  }

  /* step 7: the L-step with the Q1 Galerkin operators
   * A_x^+- = X^T T(+-1, 0) X, A_y^+- = X^T T(0, +-1) X (T the Q1 transport
   * operator of the sweep), M_t, M_s, q^ in the Q1 inner product, and the
   * inflow vectors of a unit inflow on each edge */
  double *L = (double *)malloc(sizeof(double) * r * NOm);
  if (rc == 0) {
    double *Ax[2], *Ay[2], *bE[4];
    for (int sgn = 0; sgn < 2; sgn++) {
      Ax[sgn] = (double *)calloc(r * r, sizeof(double));
      Ay[sgn] = (double *)calloc(r * r, sizeof(double));
    }
    for (int e = 0; e < 4; e++) bE[e] = (double *)calloc(r, sizeof(double));
    double *Mt = (double *)calloc(r * r, sizeof(double));
    double *Ms = (double *)calloc(r * r, sizeof(double));
    double *qh = (double *)calloc(r, sizeof(double));
    double *Tu = (double *)malloc(sizeof(double) * M4);
    for (int j = 0; j < r; j++) {
      const double *Xj = Xn + (size_t)M4 * j;
      for (int sgn = 0; sgn < 2; sgn++) {
        const double o = sgn == 0 ? 1.0 : -1.0;
        q1_transport_apply(p, o, 0.0, Xj, Tu);
        for (int i = 0; i < r; i++) {
          double t = 0;
          for (int e = 0; e < M4; e++) t += Xn[e + (size_t)M4 * i] * Tu[e];
          Ax[sgn][i + r * j] = t;
        }
        q1_transport_apply(p, 0.0, o, Xj, Tu);
        for (int i = 0; i < r; i++) {
          double t = 0;
          for (int e = 0; e < M4; e++) t += Xn[e + (size_t)M4 * i] * Tu[e];
          Ay[sgn][i + r * j] = t;
        }
      }
      for (int i = 0; i < r; i++) {
        double tt = 0, ts = 0;
        for (int e = 0; e < M4; e++) {
          double xx = Xn[e + (size_t)M4 * i] * wq[e] * Xj[e];
          tt += sig_t[e / 4] * xx;
          ts += sig_s[e / 4] * xx;
        }
        Mt[i + r * j] = tt;
        Ms[i + r * j] = ts;
      }
      double tq = 0;
      for (int c = 0; c < Nx; c++) tq += q[c] * wq[4 * c] * Xj[4 * c];
      qh[j] = tq;
      /* a unit inflow through a boundary face: (length / 2) int trace_i = length trace_i(const) */
      for (int iy = 0; iy < ny; iy++)
        for (int i = 0; i < 4; i++) {
          bE[0][j] += hy * Q1_TR_L[i][0] * Xj[4 * (iy * nx) + i];
          bE[1][j] += hy * Q1_TR_R[i][0] * Xj[4 * (iy * nx + nx - 1) + i];
        }
      for (int ix = 0; ix < nx; ix++)
        for (int i = 0; i < 4; i++) {
          bE[2][j] += hx * Q1_TR_B[i][0] * Xj[4 * ix + i];
          bE[3][j] += hx * Q1_TR_T[i][0] * Xj[4 * ((ny - 1) * nx + ix) + i];
        }
    }
    rc = lstep_solve(p, r, Ax, Ay, Mt, Ms, qh, bE, Lt0, NULL, L);
    for (int sgn = 0; sgn < 2; sgn++) { free(Ax[sgn]); free(Ay[sgn]); }
    for (int e = 0; e < 4; e++) free(bE[e]);
    free(Mt); free(Ms); free(qh); free(Tu);
  }

  /* step 8: L = S W^T (Householder QR of diag(sqrt w) L^T) */
  if (rc == 0) {
    double *Mq = (double *)malloc(sizeof(double) * NOm * r);
    double *Qm = (double *)malloc(sizeof(double) * NOm * r);
    double *Rm = (double *)malloc(sizeof(double) * r * r);
    for (int j = 0; j < r; j++)
      for (int k = 0; k < NOm; k++) Mq[k + (size_t)NOm * j] = sqrt(w[k]) * L[j + r * k];
    oracle_householder_qr(NOm, r, Mq, Qm, Rm);
    for (int j = 0; j < r; j++)
      for (int k = 0; k < NOm; k++) W[k + (size_t)NOm * j] = Qm[k + (size_t)NOm * j] / sqrt(w[k]);
    for (int i = 0; i < r; i++)
      for (int j = 0; j < r; j++) S[i + r * j] = Rm[j + r * i];
    memcpy(X, Xn, sizeof(double) * M4 * r);
    free(Mq); free(Qm); free(Rm);

    /* step 9: phi of the new factors, T from its cell average */
    double *bn = (double *)calloc(r, sizeof(double));
    double *Sb = (double *)calloc(r, sizeof(double));
    for (int j = 0; j < r; j++)
      for (int k = 0; k < NOm; k++) bn[j] += w[k] * W[k + (size_t)NOm * j];
    for (int i = 0; i < r; i++)
      for (int j = 0; j < r; j++) Sb[i] += S[i + r * j] * bn[j];
    for (int e = 0; e < M4; e++) {
      double t = 0;
      for (int i = 0; i < r; i++) t += X[e + (size_t)M4 * i] * Sb[i];
      phin[e] = t;
    }
    for (int c = 0; c < Nx; c++)
      T[c] = T[c] + p->dt * oracle_sigma_at(p, c, T[c]) * (phin[4 * c] - 4.0 * ORACLE_PI * B0[c]) / D[c];
    if (phi_out) memcpy(phi_out, phin, sizeof(double) * M4);
    free(bn); free(Sb);
  }
  free(ox); free(oy); free(oz); free(w); free(wq); free(sig_s); free(q); free(B0); free(D);
  free(sig_t); free(idx); free(WLU); free(wpiv); free(beta); free(L0); free(Psi0); free(Psi);
  free(phi); free(phin); free(src); free(Kc); free(in_x); free(in_y); free(Xn); free(R); free(A);
  free(Lt0); free(P); free(L); free(Adsa);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Diffusion synthetic acceleration (Section 4.5; reading R17).        */
/* ------------------------------------------------------------------ */

/* Penalty coefficient of F0 on faces whose normal is along x (axis 0) or y
 * (axis 1): (1/4 pi) (1/2) sum_k w_k |Om_k . n|. */
double oracle_dsa_kappa(int n_polar, int n_azim, int axis) {
  int NOm = n_polar * n_azim;
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(n_polar, n_azim, ox, oy, oz, w);
  double t = 0;
  for (int k = 0; k < NOm; k++) t += w[k] * fabs(axis == 0 ? ox[k] : oy[k]);
  free(ox); free(oy); free(oz); free(w);
  return t / (8.0 * ORACLE_PI);
}

/* The faces normal to `axis`: face f of line l (f = 0 .. n, n cells along
 * the axis) lies between cell f-1 (lo) and cell f (hi); -1 = outside. */
static void face_cells(const oracle_problem *p, int axis, int l, int f, int *lo, int *hi) {
  int nx = p->nx, ny = p->ny;
  int n = axis == 0 ? nx : ny;
  int c_lo = axis == 0 ? l * nx + (f - 1) : (f - 1) * nx + l;
  int c_hi = axis == 0 ? l * nx + f : f * nx + l;
  *lo = f > 0 ? c_lo : -1;
  *hi = f < n ? c_hi : -1;
}

/* out = A u with A = (1/3) sum_j Fbar_j^T M_t^{-1} Fbar_j + F0 + M_a, the
 * DG0 form of the diffusion operator of Section 4.5 (G_j = 0):
 *   v^T Fbar_j u = sum_faces int [[u]]_j {v},
 *   v^T F0 u     = sum_faces kappa [[u]] [[v]],
 *   M_t = h^2 diag(sigma_t), M_a = h^2 diag(sigma_a),
 * with [[u]] = u_lo - u_hi across a face (normal from lo to hi), {v} the
 * mean of the two traces, and a zero trace outside the domain. */
void oracle_dsa_apply(const oracle_problem *p, const double *sig_t,
                      const double *sig_a, const double *u, double *out) {
  int nx = p->nx, ny = p->ny, N = nx * ny;
  double hx = p->lx / nx, hy = p->ly / ny, h2 = hx * hy;
  double *g = (double *)malloc(sizeof(double) * N);
  double *z = (double *)malloc(sizeof(double) * N);
  for (int c = 0; c < N; c++) out[c] = h2 * sig_a[c] * u[c];
  for (int axis = 0; axis < 2; axis++) {
    int n = axis == 0 ? nx : ny, lines = axis == 0 ? ny : nx;
    double hf = axis == 0 ? hy : hx;  /* face length */
    double kap = oracle_dsa_kappa(p->n_polar, p->n_azim, axis);
    /* g = Fbar u */
    for (int c = 0; c < N; c++) g[c] = 0;
    for (int l = 0; l < lines; l++)
      for (int f = 0; f <= n; f++) {
        int lo, hi;
        face_cells(p, axis, l, f, &lo, &hi);
        double jump = (lo >= 0 ? u[lo] : 0.0) - (hi >= 0 ? u[hi] : 0.0);
        if (lo >= 0) g[lo] += hf * jump * 0.5;
        if (hi >= 0) g[hi] += hf * jump * 0.5;
      }
    /* z = M_t^{-1} g, then out += (1/3) Fbar^T z (the face loop transposed) */
    for (int c = 0; c < N; c++) z[c] = g[c] / (h2 * sig_t[c]);
    for (int l = 0; l < lines; l++)
      for (int f = 0; f <= n; f++) {
        int lo, hi;
        face_cells(p, axis, l, f, &lo, &hi);
        double zs = hf * 0.5 * ((lo >= 0 ? z[lo] : 0.0) + (hi >= 0 ? z[hi] : 0.0));
        if (lo >= 0) out[lo] += zs / 3.0;
        if (hi >= 0) out[hi] -= zs / 3.0;
      }
    /* F0 */
    for (int l = 0; l < lines; l++)
      for (int f = 0; f <= n; f++) {
        int lo, hi;
        face_cells(p, axis, l, f, &lo, &hi);
        double jump = (lo >= 0 ? u[lo] : 0.0) - (hi >= 0 ? u[hi] : 0.0);
        if (lo >= 0) out[lo] += kap * hf * jump;
        if (hi >= 0) out[hi] -= kap * hf * jump;
      }
  }
  free(g); free(z);
}

/* The diagonal of A by probing: A couples a cell only with cells at most two
 * apart along x or along y, so applying A to the indicator of the cells
 * with (ix mod 5, iy mod 5) fixed reads A_cc for every cell of that class. */
void oracle_dsa_diag(const oracle_problem *p, const double *sig_t,
                     const double *sig_a, double *d) {
  int nx = p->nx, ny = p->ny, N = nx * ny;
  double *e = (double *)malloc(sizeof(double) * N);
  double *Ae = (double *)malloc(sizeof(double) * N);
  for (int a = 0; a < 5; a++)
    for (int b = 0; b < 5; b++) {
      for (int c = 0; c < N; c++) e[c] = ((c % nx) % 5 == a && (c / nx) % 5 == b) ? 1.0 : 0.0;
      oracle_dsa_apply(p, sig_t, sig_a, e, Ae);
      for (int c = 0; c < N; c++)
        if (e[c] != 0.0) d[c] = Ae[c];
    }
  free(e); free(Ae);
}

static double dot(int n, const double *a, const double *b) {
  double t = 0;
  for (int i = 0; i < n; i++) t += a[i] * b[i];
  return t;
}

/* Jacobi-preconditioned conjugate gradients for A x = b (x starts at 0),
 * stopping when ||r||_2 <= tol ||b||_2 or after max_iter iterations.
 * Returns the iterations taken. */
int oracle_dsa_solve(const oracle_problem *p, const double *sig_t,
                     const double *sig_a, const double *b, double tol,
                     int max_iter, double *x) {
  int N = p->nx * p->ny;
  double *d = (double *)malloc(sizeof(double) * N);
  double *r = (double *)malloc(sizeof(double) * N);
  double *z = (double *)malloc(sizeof(double) * N);
  double *pp = (double *)malloc(sizeof(double) * N);
  double *q = (double *)malloc(sizeof(double) * N);
  oracle_dsa_diag(p, sig_t, sig_a, d);
  for (int c = 0; c < N; c++) {
    x[c] = 0;
    r[c] = b[c];
    z[c] = r[c] / d[c];
    pp[c] = z[c];
  }
  double bb = dot(N, b, b), rz = dot(N, r, z);
  int it = 0;
  while (bb > 0 && it < max_iter) {
    oracle_dsa_apply(p, sig_t, sig_a, pp, q);
    double alpha = rz / dot(N, pp, q);
    for (int c = 0; c < N; c++) {
      x[c] += alpha * pp[c];
      r[c] -= alpha * q[c];
    }
    it++;
    if (dot(N, r, r) <= tol * tol * bb) break;
    for (int c = 0; c < N; c++) z[c] = r[c] / d[c];
    double rz_new = dot(N, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (int c = 0; c < N; c++) pp[c] = z[c] + beta * pp[c];
  }
  free(d); free(r); free(z); free(pp); free(q);
  return it;
}

/* The DSA step between source iterations: phi_half (the scalar flux of the
 * sweeps at phi_old) becomes phi_half + delta with
 * A delta = M_s (phi_half - phi_old).  Returns the CG iterations. */
static int dsa_correct(const oracle_problem *p, const double *sig_t,
                       const double *sig_s, const double *phi_old,
                       double *phi_half) {
  int N = p->nx * p->ny;
  double h2 = (p->lx / p->nx) * (p->ly / p->ny);
  double *sig_a = (double *)malloc(sizeof(double) * N);
  double *b = (double *)malloc(sizeof(double) * N);
  double *delta = (double *)malloc(sizeof(double) * N);
  for (int c = 0; c < N; c++) {
    sig_a[c] = sig_t[c] - sig_s[c];
    b[c] = h2 * sig_s[c] * (phi_half[c] - phi_old[c]);
  }
  int it = oracle_dsa_solve(p, sig_t, sig_a, b, p->dsa_tol, p->dsa_max_iter, delta);
  for (int c = 0; c < N; c++) phi_half[c] += delta[c];
  free(sig_a); free(b); free(delta);
  return it;
}

/* ------------------------------------------------------------------ */
/* DSA on Q1 elements (Section 4.5 with the bilinear elements; R20).   */
/* ------------------------------------------------------------------ */

/* The DG derivative D_j (axis 0: x, 1: y) on Q1 fields as a dense n x n
 * matrix (n = 4 Nx, row 4 c + i tests basis function i of cell c), column
 * major: v^T D_j u = -sum_K int_K u dv/dx_j + sum_faces int {u} [[v]]_j,
 * with [[v]]_j = v_lo - v_hi across a face normal to axis j and a zero
 * trace outside the domain. */
void oracle_q1_deriv(const oracle_problem *p, int axis, double *Dm) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny;
  size_t n = 4 * (size_t)Nx;
  double hx = p->lx / nx, hy = p->ly / ny;
  double hf = axis == 0 ? hy : hx;  /* face length */
  const double (*tlo)[2] = axis == 0 ? Q1_TR_R : Q1_TR_T;  /* traces on the face, lo side */
  const double (*thi)[2] = axis == 0 ? Q1_TR_L : Q1_TR_B;  /* hi side */
  for (size_t e = 0; e < n * n; e++) Dm[e] = 0.0;
#define DM(row, col) Dm[(size_t)(row) + n * (size_t)(col)]
  for (int c = 0; c < Nx; c++) {
    /* volume: -int_K u dv/dx_j = -(hf / 2) int int u dv/dxi_j */
    if (axis == 0) {
      DM(4 * c + 1, 4 * c + 0) -= 0.5 * hf * 4.0;
      DM(4 * c + 3, 4 * c + 2) -= 0.5 * hf * 4.0 / 3.0;
    } else {
      DM(4 * c + 2, 4 * c + 0) -= 0.5 * hf * 4.0;
      DM(4 * c + 3, 4 * c + 1) -= 0.5 * hf * 4.0 / 3.0;
    }
  }
  int nl = axis == 0 ? nx : ny, lines = axis == 0 ? ny : nx;
  for (int l = 0; l < lines; l++)
    for (int f = 0; f <= nl; f++) {
      int lo, hi;
      face_cells(p, axis, l, f, &lo, &hi);
      /* (hf / 2) int {u} [[v]]: {u} = (u_lo + u_hi) / 2, [[v]] = v_lo - v_hi */
      for (int i = 0; i < 4; i++)
        for (int m = 0; m < 4; m++) {
          if (lo >= 0) {
            DM(4 * lo + i, 4 * lo + m) += 0.25 * hf * face_prod(tlo[i], tlo[m]);
            if (hi >= 0) DM(4 * lo + i, 4 * hi + m) += 0.25 * hf * face_prod(tlo[i], thi[m]);
          }
          if (hi >= 0) {
            if (lo >= 0) DM(4 * hi + i, 4 * lo + m) -= 0.25 * hf * face_prod(thi[i], tlo[m]);
            DM(4 * hi + i, 4 * hi + m) -= 0.25 * hf * face_prod(thi[i], thi[m]);
          }
        }
    }
#undef DM
}

/* The DSA operator on Q1 fields as a dense matrix, column major:
 * A = (1/3) sum_j D_j^T M_t^{-1} D_j + F0 + M_a (R20). */
void oracle_dsa_matrix_q1(const oracle_problem *p, const double *sig_t, const double *sig_a,
                          double *A) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny;
  size_t n = 4 * (size_t)Nx;
  double hx = p->lx / nx, hy = p->ly / ny;
  double *Dm = (double *)malloc(sizeof(double) * n * n);
  for (size_t e = 0; e < n * n; e++) A[e] = 0.0;
  for (int axis = 0; axis < 2; axis++) {
    oracle_q1_deriv(p, axis, Dm);
    /* (1/3) D^T M_t^{-1} D, M_t = diag(sigma_t wq) in the Legendre basis */
    for (size_t a = 0; a < n; a++)
      for (size_t b = 0; b < n; b++) {
        double t = 0;
        for (size_t k = 0; k < n; k++) {
          double mt = sig_t[k / 4] * hx * hy * Q1_MASS[k % 4] / 4.0;
          t += Dm[k + n * a] * Dm[k + n * b] / mt;
        }
        A[a + n * b] += t / 3.0;
      }
    /* F0: kappa (hf / 2) int [[u]] [[v]] on every face */
    double kap = oracle_dsa_kappa(p->n_polar, p->n_azim, axis);
    double hf = axis == 0 ? hy : hx;
    const double (*tlo)[2] = axis == 0 ? Q1_TR_R : Q1_TR_T;
    const double (*thi)[2] = axis == 0 ? Q1_TR_L : Q1_TR_B;
    int nl = axis == 0 ? nx : ny, lines = axis == 0 ? ny : nx;
    for (int l = 0; l < lines; l++)
      for (int f = 0; f <= nl; f++) {
        int lo, hi;
        face_cells(p, axis, l, f, &lo, &hi);
        for (int i = 0; i < 4; i++)
          for (int m = 0; m < 4; m++) {
            double k2 = kap * 0.5 * hf;
            if (lo >= 0) A[(4 * lo + i) + n * (4 * lo + m)] += k2 * face_prod(tlo[i], tlo[m]);
            if (hi >= 0) A[(4 * hi + i) + n * (4 * hi + m)] += k2 * face_prod(thi[i], thi[m]);
            if (lo >= 0 && hi >= 0) {
              A[(4 * lo + i) + n * (4 * hi + m)] -= k2 * face_prod(tlo[i], thi[m]);
              A[(4 * hi + i) + n * (4 * lo + m)] -= k2 * face_prod(thi[i], tlo[m]);
            }
          }
      }
  }
  /* M_a */
  for (size_t k = 0; k < n; k++) A[k + n * k] += sig_a[k / 4] * hx * hy * Q1_MASS[k % 4] / 4.0;
  free(Dm);
}

/* The DSA step of the Q1 SN step: phi_half += delta,
 * A delta = M_s (phi_half - phi_old), by Jacobi-preconditioned CG as in
 * R17 (dsa_tol, dsa_max_iter).  Returns the CG iterations. */
/* The Q1 diffusion matrix of the step (its coefficients sig_t and
 * sig_a = sig_t - sig_s are fixed for the whole source iteration), built
 * once and handed to every correction; the caller frees it. */
static double *dsa_matrix_q1_new(const oracle_problem *p, const double *sig_t, const double *sig_s) {
  int Nx = p->nx * p->ny;
  size_t n = 4 * (size_t)Nx;
  double *sig_a = (double *)malloc(sizeof(double) * Nx);
  for (int c = 0; c < Nx; c++) sig_a[c] = sig_t[c] - sig_s[c];
  double *A = (double *)malloc(sizeof(double) * n * n);
  oracle_dsa_matrix_q1(p, sig_t, sig_a, A);
  free(sig_a);
  return A;
}
static int dsa_correct_q1(const oracle_problem *p, const double *A, const double *sig_s,
                          const double *phi_old, double *phi_half) {
  int Nx = p->nx * p->ny;
  size_t n = 4 * (size_t)Nx;
  double hx = p->lx / p->nx, hy = p->ly / p->ny;
  double *b = (double *)malloc(sizeof(double) * n);
  double *x = (double *)calloc(n, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * n);
  double *z = (double *)malloc(sizeof(double) * n);
  double *pp = (double *)malloc(sizeof(double) * n);
  double *q = (double *)malloc(sizeof(double) * n);
  for (size_t k = 0; k < n; k++) {
    b[k] = sig_s[k / 4] * hx * hy * Q1_MASS[k % 4] / 4.0 * (phi_half[k] - phi_old[k]);
    r[k] = b[k];
    z[k] = r[k] / A[k + n * k];
    pp[k] = z[k];
  }
  double bb = dot((int)n, b, b), rz = dot((int)n, r, z);
  int it = 0;
  while (bb > 0 && it < p->dsa_max_iter) {
    for (size_t a = 0; a < n; a++) {
      double t = 0;
      for (size_t k = 0; k < n; k++) t += A[a + n * k] * pp[k];
      q[a] = t;
    }
    double alpha = rz / dot((int)n, pp, q);
    for (size_t k = 0; k < n; k++) {
      x[k] += alpha * pp[k];
      r[k] -= alpha * q[k];
    }
    it++;
    if (dot((int)n, r, r) <= p->dsa_tol * p->dsa_tol * bb) break;
    for (size_t k = 0; k < n; k++) z[k] = r[k] / A[k + n * k];
    double rz_new = dot((int)n, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (size_t k = 0; k < n; k++) pp[k] = z[k] + beta * pp[k];
  }
  for (size_t k = 0; k < n; k++) phi_half[k] += x[k];
  free(b); free(x); free(r); free(z); free(pp); free(q);
  return it;
}

/* ------------------------------------------------------------------ */
/* Dense linear algebra.                                               */
/* ------------------------------------------------------------------ */

/* LU with partial pivoting of the n x n column-major A, in place; piv[i] is
 * the row swapped into position i.  Returns -1 if a pivot is exactly 0. */
static int lu_factor(int n, double *A, int *piv) {
  for (int j = 0; j < n; j++) {
    int pr = j;
    double best = fabs(A[j + n * j]);
    for (int i = j + 1; i < n; i++)
      if (fabs(A[i + n * j]) > best) { best = fabs(A[i + n * j]); pr = i; }
    piv[j] = pr;
    if (best == 0.0) return -1;
    if (pr != j)
      for (int k = 0; k < n; k++) {
        double t = A[j + n * k]; A[j + n * k] = A[pr + n * k]; A[pr + n * k] = t;
      }
    for (int i = j + 1; i < n; i++) {
      double l = A[i + n * j] / A[j + n * j];
      A[i + n * j] = l;
      for (int k = j + 1; k < n; k++) A[i + n * k] -= l * A[j + n * k];
    }
  }
  return 0;
}

static void lu_solve_inplace(int n, const double *LU, const int *piv,
                             double *b) {
  for (int i = 0; i < n; i++) {
    double t = b[i]; b[i] = b[piv[i]]; b[piv[i]] = t;
  }
  for (int i = 0; i < n; i++)
    for (int k = 0; k < i; k++) b[i] -= LU[i + n * k] * b[k];
  for (int i = n - 1; i >= 0; i--) {
    for (int k = i + 1; k < n; k++) b[i] -= LU[i + n * k] * b[k];
    b[i] /= LU[i + n * i];
  }
}

/* Solves A Xout = B for nrhs right-hand sides (column-major). */
int oracle_lu_solve(int n, const double *A, int nrhs, const double *B,
                    double *Xout) {
  double *LU = (double *)malloc(sizeof(double) * n * n);
  int *piv = (int *)malloc(sizeof(int) * n);
  memcpy(LU, A, sizeof(double) * n * n);
  int rc = lu_factor(n, LU, piv);
  if (rc == 0) {
    memcpy(Xout, B, sizeof(double) * n * nrhs);
    for (int j = 0; j < nrhs; j++) lu_solve_inplace(n, LU, piv, Xout + n * j);
  }
  free(LU);
  free(piv);
  return rc;
}

/* Thin Householder QR, A (m x n, m >= n) = Q (m x n) R (n x n), R with a
 * non-negative diagonal.  A zero column leaves its reflector the identity,
 * so Q stays orthonormal when A is rank deficient. */
void oracle_householder_qr(int m, int n, const double *A, double *Q,
                           double *R) {
  double *V = (double *)malloc(sizeof(double) * m * n); /* reduced A */
  double *H = (double *)calloc((size_t)m * n, sizeof(double)); /* reflectors */
  double *hn = (double *)calloc(n, sizeof(double)); /* |v|^2 */
  memcpy(V, A, sizeof(double) * m * n);
  for (int j = 0; j < n; j++) {
    double nrm = 0;
    for (int i = j; i < m; i++) nrm += V[i + m * j] * V[i + m * j];
    nrm = sqrt(nrm);
    double alpha = V[j + m * j] >= 0 ? -nrm : nrm;
    for (int i = j; i < m; i++) H[i + m * j] = V[i + m * j];
    H[j + m * j] -= alpha;
    double vv = 0;
    for (int i = j; i < m; i++) vv += H[i + m * j] * H[i + m * j];
    hn[j] = vv;
    if (vv > 0) {
#pragma omp parallel for schedule(static) if ((size_t)m * (n - j) > 65536)
      for (int k = j; k < n; k++) {
        double d = 0;
        for (int i = j; i < m; i++) d += H[i + m * j] * V[i + m * k];
        double f = 2.0 * d / vv;
        for (int i = j; i < m; i++) V[i + m * k] -= f * H[i + m * j];
      }
    }
  }
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) R[i + n * j] = i <= j ? V[i + m * j] : 0.0;
  /* Q = H_0 H_1 ... H_{n-1} [I; 0] */
  for (int j = 0; j < n; j++)
    for (int i = 0; i < m; i++) Q[i + m * j] = i == j ? 1.0 : 0.0;
  for (int j = n - 1; j >= 0; j--) {
    if (hn[j] == 0) continue;
#pragma omp parallel for schedule(static) if ((size_t)m * n > 65536)
    for (int k = 0; k < n; k++) {
      double d = 0;
      for (int i = j; i < m; i++) d += H[i + m * j] * Q[i + m * k];
      double f = 2.0 * d / hn[j];
      for (int i = j; i < m; i++) Q[i + m * k] -= f * H[i + m * j];
    }
  }
  for (int j = 0; j < n; j++)
    if (R[j + n * j] < 0) {
      for (int k = 0; k < n; k++) R[j + n * k] = -R[j + n * k];
      for (int i = 0; i < m; i++) Q[i + m * j] = -Q[i + m * j];
    }
  free(V);
  free(H);
  free(hn);
}

/* One-sided (Hestenes) Jacobi SVD of the square A = U diag(s) V^T,
 * singular values descending; columns for zero singular values are
 * completed to an orthonormal basis. */
int oracle_jacobi_svd(int n, const double *A, double *U, double *s,
                      double *V) {
  double *Uw = (double *)malloc(sizeof(double) * n * n);
  double *Vw = (double *)malloc(sizeof(double) * n * n);
  memcpy(Uw, A, sizeof(double) * n * n);
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) Vw[i + n * j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    int rotated = 0;
    for (int i = 0; i < n - 1; i++)
      for (int j = i + 1; j < n; j++) {
        double al = 0, be = 0, ga = 0;
        for (int k = 0; k < n; k++) {
          al += Uw[k + n * i] * Uw[k + n * i];
          be += Uw[k + n * j] * Uw[k + n * j];
          ga += Uw[k + n * i] * Uw[k + n * j];
        }
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        rotated = 1;
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int k = 0; k < n; k++) {
          double ui = Uw[k + n * i], uj = Uw[k + n * j];
          Uw[k + n * i] = cs * ui - sn * uj;
          Uw[k + n * j] = sn * ui + cs * uj;
          double vi = Vw[k + n * i], vj = Vw[k + n * j];
          Vw[k + n * i] = cs * vi - sn * vj;
          Vw[k + n * j] = sn * vi + cs * vj;
        }
      }
    if (!rotated) break;
  }
  /* singular values and descending order (stable in the column index) */
  double *sv = (double *)malloc(sizeof(double) * n);
  int *ord = (int *)malloc(sizeof(int) * n);
  for (int j = 0; j < n; j++) {
    double t = 0;
    for (int k = 0; k < n; k++) t += Uw[k + n * j] * Uw[k + n * j];
    sv[j] = sqrt(t);
    ord[j] = j;
  }
  for (int a = 1; a < n; a++) {
    int key = ord[a], b = a - 1;
    while (b >= 0 && sv[ord[b]] < sv[key]) { ord[b + 1] = ord[b]; b--; }
    ord[b + 1] = key;
  }
  double smax = n > 0 ? sv[ord[0]] : 0.0;
  for (int j = 0; j < n; j++) {
    int o = ord[j];
    s[j] = sv[o];
    for (int k = 0; k < n; k++) V[k + n * j] = Vw[k + n * o];
    if (sv[o] > 1e-300 && sv[o] > 1e-15 * smax) {
      for (int k = 0; k < n; k++) U[k + n * j] = Uw[k + n * o] / sv[o];
    } else {
      for (int k = 0; k < n; k++) U[k + n * j] = 0.0;
      s[j] = sv[o];
    }
  }
  /* complete U columns of (numerically) zero singular values */
  for (int j = 0; j < n; j++) {
    double t = 0;
    for (int k = 0; k < n; k++) t += U[k + n * j] * U[k + n * j];
    if (t > 0.5) continue;
    for (int e = 0; e < n; e++) {
      double *u = U + n * j;
      for (int k = 0; k < n; k++) u[k] = k == e ? 1.0 : 0.0;
      for (int pass = 0; pass < 2; pass++)
        for (int l = 0; l < n; l++) {
          if (l == j) continue;
          double d = 0, ll = 0;
          for (int k = 0; k < n; k++) { d += U[k + n * l] * u[k]; ll += U[k + n * l] * U[k + n * l]; }
          if (ll < 0.5) continue;
          for (int k = 0; k < n; k++) u[k] -= d * U[k + n * l];
        }
      double nn = 0;
      for (int k = 0; k < n; k++) nn += u[k] * u[k];
      if (nn > 1e-2) {
        nn = sqrt(nn);
        for (int k = 0; k < n; k++) u[k] /= nn;
        break;
      }
    }
  }
  free(Uw);
  free(Vw);
  free(sv);
  free(ord);
  return 0;
}

/* Argmax with the tie rule of reading R8: the lowest index whose value is
 * within a relative TIE_REL of the maximum; entries with skip[k] != 0 are
 * excluded. */
static int argmax_tie(int n, const double *v, const int *skip) {
  double m = -1.0;
  for (int k = 0; k < n; k++)
    if (!(skip && skip[k]) && v[k] > m) m = v[k];
  for (int k = 0; k < n; k++)
    if (!(skip && skip[k]) && v[k] >= m * (1.0 - TIE_REL)) return k;
  return -1;
}

/* Angle selection by column-pivoted Householder QR (Businger-Golub) of the
 * r x n matrix W^T: the pivot at step s is the column of largest remaining
 * norm below row s; idx = the first r pivots. */
int oracle_qdeim(int n, int r, const double *W, int *idx) {
  double *A = (double *)malloc(sizeof(double) * r * n); /* A = W^T, r x n */
  double *nrm = (double *)malloc(sizeof(double) * n);
  int *used = (int *)calloc(n, sizeof(int));
  double *v = (double *)malloc(sizeof(double) * r);
  for (int k = 0; k < n; k++)
    for (int j = 0; j < r; j++) A[j + r * k] = W[k + n * j];
  for (int s = 0; s < r; s++) {
    for (int k = 0; k < n; k++) {
      double t = 0;
      for (int i = s; i < r; i++) t += A[i + r * k] * A[i + r * k];
      nrm[k] = sqrt(t);
    }
    int piv = argmax_tie(n, nrm, used);
    if (piv < 0) {  /* no finite column norm left: W is not finite */
      free(A); free(nrm); free(used); free(v);
      return -1;
    }
    idx[s] = piv;
    used[piv] = 1;
    /* Householder reflector zeroing A[s+1:, piv]; applied to every column */
    double alpha = A[s + r * piv] >= 0 ? -nrm[piv] : nrm[piv];
    for (int i = s; i < r; i++) v[i] = A[i + r * piv];
    v[s] -= alpha;
    double vv = 0;
    for (int i = s; i < r; i++) vv += v[i] * v[i];
    if (vv > 0)
      for (int k = 0; k < n; k++) {
        double d = 0;
        for (int i = s; i < r; i++) d += v[i] * A[i + r * k];
        double f = 2.0 * d / vv;
        for (int i = s; i < r; i++) A[i + r * k] -= f * v[i];
      }
  }
  free(A);
  free(nrm);
  free(used);
  free(v);
  return 0;
}

/* Greedy DEIM of Section 4.2: Om_1 = argmax |W_1|; then the next point
 * maximises the residual of W_j after interpolation on the points so far. */
int oracle_deim(int n, int r, const double *W, int *idx) {
  double *res = (double *)malloc(sizeof(double) * n);
  double *M = (double *)malloc(sizeof(double) * r * r);
  double *rhs = (double *)malloc(sizeof(double) * r);
  double *cf = (double *)malloc(sizeof(double) * r);
  int *used = (int *)calloc(n, sizeof(int));
  int rc = 0;
  for (int j = 0; j < r; j++) {
    for (int k = 0; k < n; k++) res[k] = W[k + n * j];
    if (j > 0) {
      /* interpolation coefficients: sum_l c_l W_l(Om_i) = W_j(Om_i) */
      for (int i = 0; i < j; i++) {
        rhs[i] = W[idx[i] + n * j];
        for (int l = 0; l < j; l++) M[i + j * l] = W[idx[i] + n * l];
      }
      if (oracle_lu_solve(j, M, 1, rhs, cf) != 0) { rc = -1; break; }
      for (int k = 0; k < n; k++)
        for (int l = 0; l < j; l++) res[k] -= cf[l] * W[k + n * l];
    }
    for (int k = 0; k < n; k++) res[k] = fabs(res[k]);
    idx[j] = argmax_tie(n, res, used);
    if (idx[j] < 0) { rc = -1; break; }  /* no finite residual left: W is not finite */
    used[idx[j]] = 1;
  }
  free(res);
  free(M);
  free(rhs);
  free(cf);
  free(used);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Initial factors (reading R11).                                      */
/* ------------------------------------------------------------------ */

/* Appends candidate vector v (length m) to the orthonormal set Q (m x *cnt)
 * under the weighted inner product sum_i wt_i a_i b_i by two passes of
 * modified Gram-Schmidt; skipped if less than 1e-8 of it survives. */
static void gs_append(int m, const double *wt, double *Q, int *cnt,
                      const double *v) {
  double *u = (double *)malloc(sizeof(double) * m);
  memcpy(u, v, sizeof(double) * m);
  double n0 = 0;
  for (int i = 0; i < m; i++) n0 += wt[i] * u[i] * u[i];
  n0 = sqrt(n0);
  if (n0 == 0) { free(u); return; }
  for (int pass = 0; pass < 2; pass++)
    for (int l = 0; l < *cnt; l++) {
      double d = 0;
      for (int i = 0; i < m; i++) d += wt[i] * Q[i + m * l] * u[i];
      for (int i = 0; i < m; i++) u[i] -= d * Q[i + m * l];
    }
  double n1 = 0;
  for (int i = 0; i < m; i++) n1 += wt[i] * u[i] * u[i];
  n1 = sqrt(n1);
  if (n1 > 1e-8 * n0) {
    for (int i = 0; i < m; i++) Q[i + m * (*cnt)] = u[i] / n1;
    (*cnt)++;
  }
  free(u);
}

/* X0: f = B(T0) first, then cos(pi k x^)cos(pi l y^) modes in (k+l, k)
 * order; W0: monomials Om_x^a Om_y^b by degree (a descending), then the
 * same times Om_z; S0 = diag(|f| sqrt(4 pi), 0, ...), so X0 S0 W0^T = f. */
int oracle_initial_factors(const oracle_problem *p, const double *T0, int r,
                           double *X0, double *S0, double *W0) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim;
  double hx = p->lx / nx, hy = p->ly / ny, h2 = hx * hy;
  if (r < 1 || r > Nx || r > NOm) return -1;
  double *wt = (double *)malloc(sizeof(double) * Nx);
  double *v = (double *)malloc(sizeof(double) * (Nx > NOm ? Nx : NOm));
  double *Q = (double *)malloc(sizeof(double) * Nx * r);
  for (int c = 0; c < Nx; c++) wt[c] = h2;
  int cnt = 0;
  double fn = 0;
  for (int c = 0; c < Nx; c++) {
    v[c] = oracle_planck(p->a_rad, p->c, T0[c]);
    fn += h2 * v[c] * v[c];
  }
  fn = sqrt(fn);
  gs_append(Nx, wt, Q, &cnt, v);
  for (int d = 0; d <= nx + ny - 2 && cnt < r; d++)
    for (int k = 0; k <= d && cnt < r; k++) {
      int l = d - k;
      if (k >= nx || l >= ny) continue;
      for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++)
          v[iy * nx + ix] = cos(ORACLE_PI * k * (ix + 0.5) / nx) *
                            cos(ORACLE_PI * l * (iy + 0.5) / ny);
      gs_append(Nx, wt, Q, &cnt, v);
    }
  if (cnt < r) { free(wt); free(v); free(Q); return -1; }
  memcpy(X0, Q, sizeof(double) * Nx * r);
  free(Q);

  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  double *QW = (double *)malloc(sizeof(double) * NOm * r);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  cnt = 0;
  for (int e = 0; e <= 1 && cnt < r; e++)
    for (int d = 0; d <= 12 && cnt < r; d++)
      for (int a = d; a >= 0 && cnt < r; a--) {
        int b = d - a;
        for (int k = 0; k < NOm; k++)
          v[k] = pow(ox[k], a) * pow(oy[k], b) * (e ? oz[k] : 1.0);
        gs_append(NOm, w, QW, &cnt, v);
      }
  int rc = cnt < r ? -1 : 0;
  if (rc == 0) memcpy(W0, QW, sizeof(double) * NOm * r);
  for (int i = 0; i < r * r; i++) S0[i] = 0.0;
  S0[0] = fn * sqrt(4.0 * ORACLE_PI);
  free(ox); free(oy); free(oz); free(w); free(QW); free(wt); free(v);
  return rc;
}

/* ------------------------------------------------------------------ */
/* L-step (Algorithm 1 step 7; Eq. L step; solution by the C-bar device */
/* of Section 3.3).                                                    */
/* ------------------------------------------------------------------ */

/* Upwind difference D^{+-} of the DG0 scheme with zero inflow (the inflow
 * value is moved to the right-hand side): dir = +1 uses the west/south
 * neighbour, -1 the east/north one.  axis 0 = x, 1 = y. */
static void upwind_diff(const oracle_problem *p, int axis, int dir,
                        const double *u, double *out) {
  int nx = p->nx, ny = p->ny;
  double h = axis == 0 ? p->lx / nx : p->ly / ny;
  for (int iy = 0; iy < ny; iy++)
    for (int ix = 0; ix < nx; ix++) {
      int jx = axis == 0 ? ix - dir : ix, jy = axis == 1 ? iy - dir : iy;
      double up = (jx >= 0 && jx < nx && jy >= 0 && jy < ny) ? u[jy * nx + jx] : 0.0;
      out[iy * nx + ix] = (u[iy * nx + ix] - up) / h;
    }
}

int oracle_lstep(const oracle_problem *p, int r, const double *X,
                 const double *sigma_t, const double *sigma_s,
                 const double *q, const double *Lt0, double *L) {
  return oracle_lstep_g(p, r, X, sigma_t, sigma_s, q, Lt0, NULL, L);
}

/* The L-step with an extra inflow vector per angle, gext (r x NOm; NULL: none). */
int oracle_lstep_g(const oracle_problem *p, int r, const double *X,
                   const double *sigma_t, const double *sigma_s,
                   const double *q, const double *Lt0, const double *gext, double *L) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim;
  double hx = p->lx / nx, hy = p->ly / ny, h2 = hx * hy;
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);

  /* Galerkin operators <D X_j, X_i>, M_t, M_s, <q, X_i>, edge sums */
  double *Ax[2], *Ay[2]; /* [0] = '+' (west/south upwind), [1] = '-' */
  for (int s = 0; s < 2; s++) {
    Ax[s] = (double *)calloc(r * r, sizeof(double));
    Ay[s] = (double *)calloc(r * r, sizeof(double));
  }
  double *Mt = (double *)calloc(r * r, sizeof(double));
  double *Ms = (double *)calloc(r * r, sizeof(double));
  double *qh = (double *)calloc(r, sizeof(double));
  double *bE[4];
  for (int e = 0; e < 4; e++) bE[e] = (double *)calloc(r, sizeof(double));
#pragma omp parallel if ((size_t)Nx * r > 65536)
  {
  double *Du = (double *)malloc(sizeof(double) * Nx);
#pragma omp for schedule(dynamic, 1)
  for (int j = 0; j < r; j++) {
    const double *Xj = X + (size_t)Nx * j;
    for (int s = 0; s < 2; s++) {
      upwind_diff(p, 0, s == 0 ? 1 : -1, Xj, Du);
      for (int i = 0; i < r; i++) {
        double t = 0;
        for (int c = 0; c < Nx; c++) t += X[c + (size_t)Nx * i] * Du[c];
        Ax[s][i + r * j] = h2 * t;
      }
      upwind_diff(p, 1, s == 0 ? 1 : -1, Xj, Du);
      for (int i = 0; i < r; i++) {
        double t = 0;
        for (int c = 0; c < Nx; c++) t += X[c + (size_t)Nx * i] * Du[c];
        Ay[s][i + r * j] = h2 * t;
      }
    }
    for (int i = 0; i < r; i++) {
      double tt = 0, ts = 0;
      for (int c = 0; c < Nx; c++) {
        double xx = X[c + (size_t)Nx * i] * Xj[c];
        tt += sigma_t[c] * xx;
        ts += sigma_s[c] * xx;
      }
      Mt[i + r * j] = h2 * tt;
      Ms[i + r * j] = h2 * ts;
    }
    double tq = 0;
    for (int c = 0; c < Nx; c++) tq += q[c] * Xj[c];
    qh[j] = h2 * tq;
    for (int iy = 0; iy < ny; iy++) {
      bE[0][j] += hy * Xj[iy * nx + 0];
      bE[1][j] += hy * Xj[iy * nx + nx - 1];
    }
    for (int ix = 0; ix < nx; ix++) {
      bE[2][j] += hx * Xj[ix];
      bE[3][j] += hx * Xj[(ny - 1) * nx + ix];
    }
  }
  free(Du);
  }

  int rc = lstep_solve(p, r, Ax, Ay, Mt, Ms, qh, bE, Lt0, gext, L);
  for (int s = 0; s < 2; s++) { free(Ax[s]); free(Ay[s]); }
  for (int e = 0; e < 4; e++) free(bE[e]);
  free(Mt); free(Ms); free(qh); free(ox); free(oy); free(oz); free(w);
  return rc;
}

/* The solve of step 7 (Eq. L step) from the Galerkin operators: per angle
 * B_k = |ox| Ax^s + |oy| Ay^s + M_t, Q_k = q^ + Lt0_k/(c dt) + the inflow
 * terms; Cbar = sum_k w_k B_k^-1, zeta = sum_k w_k B_k^-1 Q_k;
 * (I - Cbar M_s / 4 pi) Lbar = zeta; L_k = B_k^-1 (Q_k + M_s Lbar / 4 pi)
 * (the C-bar device of Section 3.3). */
static int lstep_solve(const oracle_problem *p, int r, double *const *Ax, double *const *Ay,
                       const double *Mt, const double *Ms, const double *qh,
                       double *const *bE, const double *Lt0, const double *gext, double *L) {
  int NOm = p->n_polar * p->n_azim;
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  double inv_cdt = 1.0 / (p->c * p->dt);
  double *Bk = (double *)malloc(sizeof(double) * r * r * NOm);
  double *Qk = (double *)malloc(sizeof(double) * r * NOm);
  double *Cbar = (double *)calloc(r * r, sizeof(double));
  double *zeta = (double *)calloc(r, sizeof(double));
  double *I_r = (double *)calloc(r * r, sizeof(double));
  /* B_k^-1 and B_k^-1 Q_k of every angle first (independent per angle),
   * then the sums over angles in angle order */
  double *Binv_all = (double *)malloc(sizeof(double) * r * r * NOm);
  double *BQ_all = (double *)malloc(sizeof(double) * r * NOm);
  int *rck = (int *)calloc(NOm, sizeof(int));
  for (int i = 0; i < r; i++) I_r[i + r * i] = 1.0;
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 8) if (NOm * r * r > 65536)
  for (int k = 0; k < NOm; k++) {
    int sx = ox[k] > 0 ? 0 : 1, sy = oy[k] > 0 ? 0 : 1;
    double *B = Bk + (size_t)r * r * k;
    for (int e = 0; e < r * r; e++)
      B[e] = fabs(ox[k]) * Ax[sx][e] + fabs(oy[k]) * Ay[sy][e] + Mt[e];
    double *Q = Qk + (size_t)r * k;
    /* a reflective edge's inflow comes in through gext (reading R19) */
    int ex = ox[k] > 0 ? 0 : 1, ey = oy[k] > 0 ? 2 : 3;
    double psx = p->reflect[ex] ? 0.0 : p->psi_edge[ex];
    double psy = p->reflect[ey] ? 0.0 : p->psi_edge[ey];
    const double *bx = ox[k] > 0 ? bE[0] : bE[1];
    const double *by = oy[k] > 0 ? bE[2] : bE[3];
    for (int i = 0; i < r; i++)
      Q[i] = qh[i] + inv_cdt * Lt0[i + r * k] + fabs(ox[k]) * psx * bx[i] +
             fabs(oy[k]) * psy * by[i] +
             (gext ? gext[i + (size_t)r * k] : 0.0);
    double *Binv = Binv_all + (size_t)r * r * k, *BQ = BQ_all + (size_t)r * k;
    rck[k] = oracle_lu_solve(r, B, r, I_r, Binv);
    if (rck[k] == 0) rck[k] = oracle_lu_solve(r, B, 1, Q, BQ);
  }
  for (int k = 0; k < NOm && rc == 0; k++) {
    rc = rck[k];
    if (rc) break;
    const double *Binv = Binv_all + (size_t)r * r * k, *BQ = BQ_all + (size_t)r * k;
    for (int e = 0; e < r * r; e++) Cbar[e] += w[k] * Binv[e];
    for (int i = 0; i < r; i++) zeta[i] += w[k] * BQ[i];
  }
  /* (I - Cbar Ms / 4pi) Lbar = zeta;  L_k = B_k^{-1} (Q_k + Ms Lbar / 4pi) */
  double *Msys = (double *)malloc(sizeof(double) * r * r);
  double *Lbar = (double *)malloc(sizeof(double) * r);
  double *rhs = (double *)malloc(sizeof(double) * r);
  if (rc == 0) {
    for (int i = 0; i < r; i++)
      for (int j = 0; j < r; j++) {
        double t = 0;
        for (int l = 0; l < r; l++) t += Cbar[i + r * l] * Ms[l + r * j];
        Msys[i + r * j] = (i == j ? 1.0 : 0.0) - t / (4.0 * ORACLE_PI);
      }
    rc = oracle_lu_solve(r, Msys, 1, zeta, Lbar);
  }
  if (rc == 0) {
    /* M_s Lbar / 4 pi is the same for every angle */
    for (int i = 0; i < r; i++) {
      double t = 0;
      for (int l = 0; l < r; l++) t += Ms[i + r * l] * Lbar[l];
      rhs[i] = t / (4.0 * ORACLE_PI);
    }
#pragma omp parallel for schedule(dynamic, 8) if (NOm * r * r > 65536)
    for (int k = 0; k < NOm; k++) {
      double *rk = (double *)malloc(sizeof(double) * r);
      for (int i = 0; i < r; i++) rk[i] = Qk[i + (size_t)r * k] + rhs[i];
      rck[k] = oracle_lu_solve(r, Bk + (size_t)r * r * k, 1, rk, L + (size_t)r * k);
      free(rk);
    }
    for (int k = 0; k < NOm && rc == 0; k++) rc = rck[k];
  }
  free(Bk); free(Qk); free(Cbar); free(zeta); free(I_r); free(Binv_all); free(BQ_all); free(rck);
  free(Msys); free(Lbar); free(rhs); free(ox); free(oy); free(oz); free(w);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Energy bookkeeping (Section 2.1: d/dt[rho_cv T + phi/c] + div F = 0). */
/* ------------------------------------------------------------------ */

static double energy(const oracle_problem *p, const double *T,
                     const double *phi) {
  int Nx = p->nx * p->ny;
  double h2 = (p->lx / p->nx) * (p->ly / p->ny), E = 0;
  for (int c = 0; c < Nx; c++) E += h2 * (p->rho_cv[c] * T[c] + phi[c] / p->c);
  return E;
}

/* Boundary energy rates for angular values psi(c, k) = get(c, k): outflow
 * uses the upwind (cell) value, inflow the prescribed edge value. */
typedef double (*psi_getter)(const void *ctx, int c, int k);
static void boundary_rates(const oracle_problem *p, const double *ox,
                           const double *oy, const double *w, psi_getter get,
                           const void *ctx, double *out, double *in) {
  int nx = p->nx, ny = p->ny, NOm = p->n_polar * p->n_azim;
  double hx = p->lx / nx, hy = p->ly / ny;
  double o = 0, i_ = 0;
  for (int k = 0; k < NOm; k++) {
    for (int iy = 0; iy < ny; iy++) { /* left (n = -x) and right (n = +x) */
      if (ox[k] < 0) o += w[k] * (-ox[k]) * hy * get(ctx, iy * nx, k);
      else i_ += w[k] * ox[k] * hy * p->psi_edge[0];
      if (ox[k] > 0) o += w[k] * ox[k] * hy * get(ctx, iy * nx + nx - 1, k);
      else i_ += w[k] * (-ox[k]) * hy * p->psi_edge[1];
    }
    for (int ix = 0; ix < nx; ix++) { /* bottom (n = -y) and top (n = +y) */
      if (oy[k] < 0) o += w[k] * (-oy[k]) * hx * get(ctx, ix, k);
      else i_ += w[k] * oy[k] * hx * p->psi_edge[2];
      if (oy[k] > 0) o += w[k] * oy[k] * hx * get(ctx, (ny - 1) * nx + ix, k);
      else i_ += w[k] * (-oy[k]) * hx * p->psi_edge[3];
    }
  }
  *out = o;
  *in = i_;
}

typedef struct { const double *X, *L; int Nx, r; } xl_ctx;
static double get_xl(const void *ctx, int c, int k) {
  const xl_ctx *g = (const xl_ctx *)ctx;
  double t = 0;
  for (int i = 0; i < g->r; i++) t += g->X[c + (size_t)g->Nx * i] * g->L[i + g->r * k];
  return t;
}

/* phi_c = sum_k w_k psi(c, Om_k) = sum_ij X_ci S_ij beta_j, beta_j = sum_k w_k W_kj */
static void phi_from_factors(int Nx, int NOm, int r, const double *X,
                             const double *S, const double *W,
                             const double *w, double *phi) {
  double *beta = (double *)calloc(r, sizeof(double));
  double *Sb = (double *)calloc(r, sizeof(double));
  for (int j = 0; j < r; j++)
    for (int k = 0; k < NOm; k++) beta[j] += w[k] * W[k + (size_t)NOm * j];
  for (int i = 0; i < r; i++)
    for (int j = 0; j < r; j++) Sb[i] += S[i + r * j] * beta[j];
#pragma omp parallel for schedule(static) if (Nx > 16384)
  for (int c = 0; c < Nx; c++) {
    double t = 0;
    for (int i = 0; i < r; i++) t += X[c + (size_t)Nx * i] * Sb[i];
    phi[c] = t;
  }
  free(beta);
  free(Sb);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 steps 3-4: collocation sweeps with source iteration.    */
/* ------------------------------------------------------------------ */

/* psi0_j(x) = sum_k L0_k(Om^(j)) X0_k(x) (step 3); then the fixed-point
 * iteration of Eq. (steady state collocation): with phi = beta^T What^{-1}
 * Psi, sweep every chosen angle against
 *   src_j = sigma_s phi / (4 pi) + q + psi0_j / (c dt)
 * and repeat until max|phi_new - phi| <= tol max|phi_new| (reading R7);
 * phi starts from the old state at the chosen angles.  With fixed > 0,
 * exactly `fixed` iterations.  Psi is the last sweep's output. */
/* For boundary cell c with kappa = What^-1 Psi(c) (the coefficients of
 * psi(c, .) in W0): the inflow of every chosen angle entering a reflective
 * edge through c, psi(c, Om_R) = sum_m W0[R, m] kappa_m with R the mirror
 * angle (reading R19). */
static void reflected_inflow(const oracle_problem *p, int r, const int *idx, const double *ox,
                             const double *oy, const double *W, int NOm, int c,
                             const double *kappa, double *in_x, double *in_y) {
  int nx = p->nx, ny = p->ny, ix = c % nx, iy = c / nx;
  for (int j = 0; j < r; j++) {
    int k = idx[j], ex = ox[k] > 0 ? 0 : 1, ey = oy[k] > 0 ? 2 : 3;
    if (p->reflect[ex] && ix == (ex == 0 ? 0 : nx - 1)) {
      int km = oracle_reflect_index(p->n_polar, p->n_azim, k, 0);
      double t = 0;
      for (int m = 0; m < r; m++) t += W[km + (size_t)NOm * m] * kappa[m];
      in_x[j * ny + iy] = t;
    }
    if (p->reflect[ey] && iy == (ey == 2 ? 0 : ny - 1)) {
      int km = oracle_reflect_index(p->n_polar, p->n_azim, k, 1);
      double t = 0;
      for (int m = 0; m < r; m++) t += W[km + (size_t)NOm * m] * kappa[m];
      in_y[j * nx + ix] = t;
    }
  }
}

/* Relaxation of the collocation source iteration (reading R22): the
 * iteration phi <- phi + omega (phi^{l+1/2} - phi) starts with omega = 1
 * (plain source iteration); each time the sweeps' change max|phi^{l+1/2} -
 * phi| has grown by more than RELAX_GROW for RELAX_RUN consecutive
 * iterations while above RELAX_MIN max|phi^{l+1/2}|, omega is halved, down
 * to RELAX_FLOOR; a further such run means the relaxed iteration diverges
 * too, and the step ends as not converged (returns 1).  The fixed point and
 * the stopping test are unchanged; only a growing (diverging) iteration is
 * affected.  The omega of an update is the one decided after the previous
 * iteration. */
#define RELAX_GROW 1.05
#define RELAX_MIN 1e-4
#define RELAX_RUN 3
#define RELAX_FLOOR 0.125
static int relax_track(double dmax, double pmax, double *dprev, int *grow, double *omega) {
  int give_up = 0;
  if (*dprev >= 0 && dmax > RELAX_GROW * *dprev && dmax > RELAX_MIN * pmax) {
    if (++*grow >= RELAX_RUN) {
      if (*omega <= RELAX_FLOOR) give_up = 1;
      *omega *= 0.5;
      *grow = 0;
    }
  } else {
    *grow = 0;
  }
  *dprev = dmax;
  return give_up;
}

static int collocation_si(const oracle_problem *p, int r, const double *X0,
                          const double *L0, const int *idx, const double *WLU,
                          const int *wpiv, const double *beta, const double *ox,
                          const double *oy, const double *sig_t,
                          const double *sig_s, const double *q, double tol,
                          int max_iter, int fixed, double *Psi, int *iters_out,
                          int *dsa_iters_out, const double *W) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim;
  double inv_cdt = 1.0 / (p->c * p->dt);
  /* inflow per chosen angle and boundary row (x-edge) or column (y-edge);
   * on a reflective edge (reading R19) the mirror direction's value
   * W0(Om_R)^T What^-1 Psi in the boundary cell, from the previous
   * iteration (psi0 in the first) */
  const int refl = p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3];
  double *in_x = (double *)malloc(sizeof(double) * r * ny);
  double *in_y = (double *)malloc(sizeof(double) * r * nx);
  for (int j = 0; j < r; j++) {
    for (int iy = 0; iy < ny; iy++) in_x[j * ny + iy] = inflow_x(p, ox[idx[j]]);
    for (int ix = 0; ix < nx; ix++) in_y[j * nx + ix] = inflow_y(p, oy[idx[j]]);
  }
  double *Psi0 = (double *)malloc(sizeof(double) * Nx * r);
  double *phi = (double *)malloc(sizeof(double) * Nx);
  double *phin = (double *)malloc(sizeof(double) * Nx);
  double *src = (double *)malloc(sizeof(double) * Nx);
  const int par = (size_t)Nx * r > 65536;
#pragma omp parallel for schedule(static) if (par)
  for (int j = 0; j < r; j++)
    for (int c = 0; c < Nx; c++) {
      double t = 0;
      for (int k = 0; k < r; k++) t += L0[k + r * idx[j]] * X0[c + (size_t)Nx * k];
      Psi0[c + (size_t)Nx * j] = t;
    }
#pragma omp parallel if (par && !refl)
  {
    double *Kc = (double *)malloc(sizeof(double) * r);
#pragma omp for schedule(static)
    for (int c = 0; c < Nx; c++) {
      for (int j = 0; j < r; j++) Kc[j] = Psi0[c + (size_t)Nx * j];
      lu_solve_inplace(r, WLU, wpiv, Kc);
      double t = 0;
      for (int j = 0; j < r; j++) t += beta[j] * Kc[j];
      phi[c] = t;
      if (refl) reflected_inflow(p, r, idx, ox, oy, W, NOm, c, Kc, in_x, in_y);
    }
    free(Kc);
  }
  int cap = fixed > 0 ? fixed : max_iter;
  int iters = 0, converged = 0, dsa_iters = 0;
  double omega = 1.0, dprev = -1.0;  /* relaxation state (reading R22) */
  int grow = 0;
  while (iters < cap) {
#pragma omp parallel if (par)
    {
      double *srcj = (double *)malloc(sizeof(double) * Nx);
#pragma omp for schedule(dynamic, 1)
      for (int j = 0; j < r; j++) {
        for (int c = 0; c < Nx; c++)
          srcj[c] = sig_s[c] * phi[c] / (4.0 * ORACLE_PI) + q[c] +
                    inv_cdt * Psi0[c + (size_t)Nx * j];
        oracle_sweep_in(p, ox[idx[j]], oy[idx[j]], sig_t, srcj, in_x + (size_t)j * ny,
                        in_y + (size_t)j * nx, Psi + (size_t)Nx * j);
      }
      free(srcj);
    }
    iters++;
    double dmax = 0, pmax = 0;
    int bad = 0;  /* a non-finite scalar flux: the iteration diverged */
#pragma omp parallel if (par && !refl) reduction(max : dmax, pmax) reduction(|| : bad)
    {
      double *Kc = (double *)malloc(sizeof(double) * r);
#pragma omp for schedule(static)
      for (int c = 0; c < Nx; c++) {
        for (int j = 0; j < r; j++) Kc[j] = Psi[c + (size_t)Nx * j];
        lu_solve_inplace(r, WLU, wpiv, Kc);
        double t = 0;
        for (int j = 0; j < r; j++) t += beta[j] * Kc[j];
        phin[c] = t;
        if (refl) reflected_inflow(p, r, idx, ox, oy, W, NOm, c, Kc, in_x, in_y);
        if (!isfinite(t)) bad = 1;
        if (fabs(t - phi[c]) > dmax) dmax = fabs(t - phi[c]);
        if (fabs(t) > pmax) pmax = fabs(t);
      }
      free(Kc);
    }
    if (bad) break;
    if (p->dsa) {
      dsa_iters += dsa_correct(p, sig_t, sig_s, phi, phin);
      memcpy(phi, phin, sizeof(double) * Nx);
    } else {
      if (omega == 1.0) memcpy(phi, phin, sizeof(double) * Nx);
      else
        for (int c = 0; c < Nx; c++) phi[c] += omega * (phin[c] - phi[c]);
      if (relax_track(dmax, pmax, &dprev, &grow, &omega)) break;
    }
    if (fixed <= 0 && dmax <= tol * pmax) { converged = 1; break; }
  }
  *iters_out = iters;
  if (dsa_iters_out) *dsa_iters_out = dsa_iters;
  free(Psi0); free(phi); free(phin); free(src); free(in_x); free(in_y);
  return (fixed <= 0 && !converged) ? -2 : 0;
}

int oracle_collocation(const oracle_problem *p, int r, const double *X0,
                       const double *S0, const double *W0, const double *T0,
                       const int *idx, double tol, int max_iter, int fixed,
                       double *Psi, int *iters) {
  int Nx = p->nx * p->ny, NOm = p->n_polar * p->n_azim;
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  double *sig_s = (double *)malloc(sizeof(double) * Nx);
  double *q = (double *)malloc(sizeof(double) * Nx);
  double *sig_t = (double *)malloc(sizeof(double) * Nx);
  double *WLU = (double *)malloc(sizeof(double) * r * r);
  int *wpiv = (int *)malloc(sizeof(int) * r);
  double *beta = (double *)calloc(r, sizeof(double));
  double *L0 = (double *)malloc(sizeof(double) * r * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  oracle_coefficients(p, T0, sig_s, q, NULL, NULL);
  for (int c = 0; c < Nx; c++) sig_t[c] = oracle_sigma_at(p, c, T0[c]) + 1.0 / (p->c * p->dt);
  for (int i = 0; i < r; i++)
    for (int j = 0; j < r; j++) WLU[i + r * j] = W0[idx[i] + (size_t)NOm * j];
  for (int j = 0; j < r; j++)
    for (int k = 0; k < NOm; k++) beta[j] += w[k] * W0[k + (size_t)NOm * j];
  for (int i = 0; i < r; i++)
    for (int k = 0; k < NOm; k++) {
      double t = 0;
      for (int l = 0; l < r; l++) t += S0[i + r * l] * W0[k + (size_t)NOm * l];
      L0[i + r * k] = t;
    }
  int rc = lu_factor(r, WLU, wpiv);
  if (rc == 0)
    rc = collocation_si(p, r, X0, L0, idx, WLU, wpiv, beta, ox, oy, sig_t, sig_s, q,
                        tol, max_iter, fixed, Psi, iters, NULL, W0);
  free(ox); free(oy); free(oz); free(w); free(sig_s); free(q); free(sig_t);
  free(WLU); free(wpiv); free(beta); free(L0);
  return rc;
}

/* Boundary entry o of a direction (ox, oy): o < ny the row of the x-edge it
 * enters, o >= ny the column of its y-edge.  Sets *c to the boundary cell
 * and returns whether that edge is reflective. */
static int refl_entry(const oracle_problem *p, double ox, double oy, int o, int *c) {
  int nx = p->nx, ny = p->ny;
  if (o < ny) {
    int ex = ox > 0 ? 0 : 1;
    *c = o * nx + (ex == 0 ? 0 : nx - 1);
    return p->reflect[ex];
  }
  int ey = oy > 0 ? 2 : 3;
  *c = (ey == 2 ? 0 : ny - 1) * nx + (o - ny);
  return p->reflect[ey];
}

/* Step 7 with reflective edges (reading R19).  The inflow of angle k
 * through a reflective edge is the value of its mirror angle R(k) in the
 * same boundary cell, which the L-step determines itself: a fixed point on
 * those boundary values, started from the collocation fluxes interpolated
 * to the mirror angles (W0(Om_R)^T What^-1 Psi), each pass an L-step with
 * the current values as an extra inflow vector, the values then taken from
 * its solution (psi(c, Om_R) = X(c) L_R), until they change by at most
 * 1e-14 relative to their size (at most 5000 passes; -2 otherwise). */
static int lstep_reflective(const oracle_problem *p, int r, const double *X,
                            const double *sig_t, const double *sig_s, const double *q,
                            const double *Lt0, const double *Psi, const double *WLU,
                            const int *wpiv, const double *W0, double *L) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim, LB = nx + ny;
  double hx = p->lx / nx, hy = p->ly / ny;
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  /* data[k LB + o]: o < ny the x-edge row o angle k enters, o >= ny the y-edge column */
  double *data = (double *)calloc((size_t)NOm * LB, sizeof(double));
  double *gext = (double *)malloc(sizeof(double) * r * NOm);
  double *kap = (double *)malloc(sizeof(double) * r);
  int rc = -2;
  for (int k = 0; k < NOm; k++)
    for (int o = 0; o < LB; o++) {
      int c;
      if (!refl_entry(p, ox[k], oy[k], o, &c)) continue;
      for (int m = 0; m < r; m++) kap[m] = Psi[c + (size_t)Nx * m];
      lu_solve_inplace(r, WLU, wpiv, kap);
      int km = oracle_reflect_index(p->n_polar, p->n_azim, k, o < ny ? 0 : 1);
      double t = 0;
      for (int m = 0; m < r; m++) t += W0[km + (size_t)NOm * m] * kap[m];
      data[(size_t)k * LB + o] = t;
    }
  for (int pass = 0; pass < 5000; pass++) {
    for (size_t e = 0; e < (size_t)r * NOm; e++) gext[e] = 0.0;
    for (int k = 0; k < NOm; k++)
      for (int o = 0; o < LB; o++) {
        int c;
        if (!refl_entry(p, ox[k], oy[k], o, &c)) continue;
        double f = o < ny ? fabs(ox[k]) * hy : fabs(oy[k]) * hx;
        for (int i = 0; i < r; i++) gext[i + (size_t)r * k] += f * X[c + (size_t)Nx * i] * data[(size_t)k * LB + o];
      }
    int lrc = oracle_lstep_g(p, r, X, sig_t, sig_s, q, Lt0, gext, L);
    if (lrc) { rc = lrc; break; }
    double dmax = 0, vmax = 0;
    for (int k = 0; k < NOm; k++)
      for (int o = 0; o < LB; o++) {
        int c;
        if (!refl_entry(p, ox[k], oy[k], o, &c)) continue;
        int km = oracle_reflect_index(p->n_polar, p->n_azim, k, o < ny ? 0 : 1);
        double t = 0;
        for (int i = 0; i < r; i++) t += X[c + (size_t)Nx * i] * L[i + (size_t)r * km];
        double d = fabs(t - data[(size_t)k * LB + o]);
        if (d > dmax) dmax = d;
        if (fabs(t) > vmax) vmax = fabs(t);
        data[(size_t)k * LB + o] = t;
      }
    if (dmax <= 1e-14 * vmax) { rc = 0; break; }
  }
  free(ox); free(oy); free(oz); free(w); free(data); free(gext); free(kap);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: one SN-like DLR time step.                             */
/* ------------------------------------------------------------------ */

int oracle_dlr_step(const oracle_problem *p, int r, double *X, double *S,
                    double *W, double *T, const oracle_dlr_opts *opt,
                    int *idx_out, double *phi_out, oracle_dlr_diag *diag) {
  int nx = p->nx, ny = p->ny, Nx = nx * ny, NOm = p->n_polar * p->n_azim;
  double hx = p->lx / nx, hy = p->ly / ny, h2 = hx * hy, h = sqrt(h2);
  double inv_cdt = 1.0 / (p->c * p->dt);
  if (r < 1 || r > Nx || r > NOm) return -1;
  const int aug = opt && opt->augment;
  if (aug && (p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3])) return -1;
  /* rank of steps 5-8: 2r for the augmented step (R15) */
  const int m = aug ? 2 * r : r;
  if (m > Nx || m > NOm) return -1;
  int rc = 0;

  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);

  double *phi0 = (double *)malloc(sizeof(double) * Nx);
  phi_from_factors(Nx, NOm, r, X, S, W, w, phi0);
  double E_before = energy(p, T, phi0);

  /* Step 1: effective scattering and source from T0 (Eqs. effective
   * scattering / effective source, reading R1). */
  double *sig_s = (double *)malloc(sizeof(double) * Nx);
  double *q = (double *)malloc(sizeof(double) * Nx);
  double *B0 = (double *)malloc(sizeof(double) * Nx);
  double *D = (double *)malloc(sizeof(double) * Nx);
  double *sig_t = (double *)malloc(sizeof(double) * Nx);
  oracle_coefficients(p, T, sig_s, q, B0, D);
  for (int c = 0; c < Nx; c++) sig_t[c] = oracle_sigma_at(p, c, T[c]) + inv_cdt;

  /* Step 2: select r angles from W0 (Section 4.2; reading R8). */
  int *idx = (int *)calloc(r, sizeof(int)); /* valid indices even if the choice fails */
  if (opt && opt->forced_idx) memcpy(idx, opt->forced_idx, sizeof(int) * r);
  else if (opt && opt->selection == 1) rc = oracle_deim(NOm, r, W, idx);
  else rc = oracle_qdeim(NOm, r, W, idx);
  if (idx_out) memcpy(idx_out, idx, sizeof(int) * r);

  /* What_ij = W0_j(Om^(i)), beta_j = int W0_j (Section 4.1) */
  double *What = (double *)malloc(sizeof(double) * r * r);
  double *WLU = (double *)malloc(sizeof(double) * r * r);
  int *wpiv = (int *)malloc(sizeof(int) * r);
  double *beta = (double *)calloc(r, sizeof(double));
  for (int i = 0; i < r; i++)
    for (int j = 0; j < r; j++) What[i + r * j] = W[idx[i] + (size_t)NOm * j];
  for (int j = 0; j < r; j++)
    for (int k = 0; k < NOm; k++) beta[j] += w[k] * W[k + (size_t)NOm * j];
  memcpy(WLU, What, sizeof(double) * r * r);
  if (rc == 0 && lu_factor(r, WLU, wpiv) != 0) rc = -1;

  /* Steps 3-4: initial condition at the chosen angles and source
   * iteration on the collocation system. */
  double *L0 = (double *)malloc(sizeof(double) * r * NOm);
  for (int i = 0; i < r; i++)
    for (int k = 0; k < NOm; k++) {
      double t = 0;
      for (int l = 0; l < r; l++) t += S[i + r * l] * W[k + (size_t)NOm * l];
      L0[i + r * k] = t;
    }
  double *Psi = (double *)malloc(sizeof(double) * Nx * r);
  int iters = 0, dsa_iters = 0;
  if (rc == 0) {
    int fixed = opt ? opt->si_fixed_iters : 0;
    rc = collocation_si(p, r, X, L0, idx, WLU, wpiv, beta, ox, oy, sig_t, sig_s, q,
                        opt ? opt->si_tol : 1e-13, opt ? opt->si_max_iter : 1000,
                        fixed, Psi, &iters, &dsa_iters, W);
  }

  /* Step 5: Psi = X R with h^2 X^T X = I (Householder QR of h Psi); the
   * augmented step (R15) factors h [Psi, X0] instead. */
  double *Xn = (double *)malloc(sizeof(double) * Nx * m);
  double *R = (double *)malloc(sizeof(double) * m * m);
  double *A = (double *)malloc(sizeof(double) * Nx * m);
  double rdr = 0;
  if (rc == 0) {
    for (size_t e = 0; e < (size_t)Nx * r; e++) A[e] = h * Psi[e];
    if (aug)
      for (size_t e = 0; e < (size_t)Nx * r; e++) A[(size_t)Nx * r + e] = h * X[e];
    oracle_householder_qr(Nx, m, A, Xn, R);
    for (size_t e = 0; e < (size_t)Nx * m; e++) Xn[e] /= h;
    double rmin = INFINITY, rmax = 0;
    for (int j = 0; j < m; j++) {
      double d = fabs(R[j + m * j]);
      if (d < rmin) rmin = d;
      if (d > rmax) rmax = d;
    }
    rdr = rmax > 0 ? rmin / rmax : 0;
  }

  /* Step 6: Lt0 = <psi0, X_j> = P L0, P_ji = h^2 <X_j, X0_i> (m x r). */
  double *P = (double *)malloc(sizeof(double) * m * r);
  double *Lt0 = (double *)malloc(sizeof(double) * m * NOm);
  if (rc == 0) {
#pragma omp parallel for collapse(2) schedule(dynamic, 1) if ((size_t)Nx * m > 65536)
    for (int jj = 0; jj < m; jj++)
      for (int i = 0; i < r; i++) {
        double t = 0;
        for (int c = 0; c < Nx; c++) t += Xn[c + (size_t)Nx * jj] * X[c + (size_t)Nx * i];
        P[jj + m * i] = h2 * t;
      }
    for (int jj = 0; jj < m; jj++)
      for (int k = 0; k < NOm; k++) {
        double t = 0;
        for (int i = 0; i < r; i++) t += P[jj + m * i] * L0[i + r * k];
        Lt0[jj + m * k] = t;
      }
  }

  /* Step 7: L-step (Eq. L step) on the m basis functions. */
  double *L = (double *)malloc(sizeof(double) * m * NOm);
  if (rc == 0) {
    if (p->reflect[0] || p->reflect[1] || p->reflect[2] || p->reflect[3])
      rc = lstep_reflective(p, m, Xn, sig_t, sig_s, q, Lt0, Psi, WLU, wpiv, W, L);
    else
      rc = oracle_lstep(p, m, Xn, sig_t, sig_s, q, Lt0, L);
  }

  /* Step 8: L = S W^T with sum_k w_k W_ki W_kj = delta: Householder QR of
   * diag(sqrt w) L^T = Q R, W = diag(1/sqrt w) Q, S = R^T; then optionally
   * S = U Sigma V^T -> X U, Sigma, W V (signs: max-|.| entry of W_j > 0).
   * The augmented step (R15) works at rank m = 2r here and keeps the r
   * largest singular values (always canonical). */
  double *Wn = (double *)malloc(sizeof(double) * NOm * m);
  double *Sn = (double *)malloc(sizeof(double) * m * m);
  if (rc == 0) {
    double *M = (double *)malloc(sizeof(double) * NOm * m);
    double *Qm = (double *)malloc(sizeof(double) * NOm * m);
    double *Rm = (double *)malloc(sizeof(double) * m * m);
    for (int j = 0; j < m; j++)
      for (int k = 0; k < NOm; k++) M[k + (size_t)NOm * j] = sqrt(w[k]) * L[j + m * k];
    oracle_householder_qr(NOm, m, M, Qm, Rm);
    for (int j = 0; j < m; j++)
      for (int k = 0; k < NOm; k++) Wn[k + (size_t)NOm * j] = Qm[k + (size_t)NOm * j] / sqrt(w[k]);
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) Sn[i + m * j] = Rm[j + m * i];
    if (aug || !opt || opt->canonicalize) {
      double *U = (double *)malloc(sizeof(double) * m * m);
      double *V = (double *)malloc(sizeof(double) * m * m);
      double *sv = (double *)malloc(sizeof(double) * m);
      oracle_jacobi_svd(m, Sn, U, sv, V);
      double *Xr = (double *)malloc(sizeof(double) * Nx * r);
      double *Wr = (double *)malloc(sizeof(double) * NOm * r);
      double *absw = (double *)malloc(sizeof(double) * NOm);
      for (int j = 0; j < r; j++) {
#pragma omp parallel for schedule(static) if (Nx > 16384)
        for (int c = 0; c < Nx; c++) {
          double t = 0;
          for (int i = 0; i < m; i++) t += Xn[c + (size_t)Nx * i] * U[i + m * j];
          Xr[c + (size_t)Nx * j] = t;
        }
        for (int k = 0; k < NOm; k++) {
          double t = 0;
          for (int i = 0; i < m; i++) t += Wn[k + (size_t)NOm * i] * V[i + m * j];
          Wr[k + (size_t)NOm * j] = t;
        }
        /* sign: the entry of largest magnitude (tie rule R8) is > 0 */
        for (int k = 0; k < NOm; k++) absw[k] = fabs(Wr[k + (size_t)NOm * j]);
        int am = argmax_tie(NOm, absw, NULL);
        if (Wr[am + (size_t)NOm * j] < 0) {
          for (int k = 0; k < NOm; k++) Wr[k + (size_t)NOm * j] = -Wr[k + (size_t)NOm * j];
          for (int c = 0; c < Nx; c++) Xr[c + (size_t)Nx * j] = -Xr[c + (size_t)Nx * j];
        }
      }
      memcpy(Xn, Xr, sizeof(double) * Nx * r);
      memcpy(Wn, Wr, sizeof(double) * NOm * r);
      for (int e = 0; e < r * r; e++) Sn[e] = 0.0;
      for (int j = 0; j < r; j++) Sn[j + r * j] = sv[j];
      free(U); free(V); free(sv); free(Xr); free(Wr); free(absw);
    }
    free(M); free(Qm); free(Rm);
  }

  /* Step 9: temperature update (Eq. temperature update, reading R1/R12). */
  if (rc == 0) {
    double *phin2 = (double *)malloc(sizeof(double) * Nx);
    phi_from_factors(Nx, NOm, r, Xn, Sn, Wn, w, phin2);
    double *Tn = (double *)malloc(sizeof(double) * Nx);
    double minT = INFINITY, minphi = INFINITY;
    for (int c = 0; c < Nx; c++) {
      Tn[c] = T[c] + p->dt * oracle_sigma_at(p, c, T[c]) * (phin2[c] - 4.0 * ORACLE_PI * B0[c]) / D[c];
      if (Tn[c] < minT) minT = Tn[c];
      if (phin2[c] < minphi) minphi = phin2[c];
    }
    if (diag) {
      xl_ctx g = {Xn, NULL, Nx, r};
      double *Lc = (double *)malloc(sizeof(double) * r * NOm);
      for (int i = 0; i < r; i++)
        for (int k = 0; k < NOm; k++) {
          double t = 0;
          for (int j = 0; j < r; j++) t += Sn[i + r * j] * Wn[k + (size_t)NOm * j];
          Lc[i + r * k] = t;
        }
      g.L = Lc;
      double out, in;
      boundary_rates(p, ox, oy, w, get_xl, &g, &out, &in);
      free(Lc);
      diag->iters = iters;
      diag->dsa_iters = dsa_iters;
      diag->E_before = E_before;
      diag->E_after = energy(p, Tn, phin2);
      diag->outflow = out;
      diag->inflow = in;
      diag->residual = diag->E_after - E_before + p->dt * (out - in);
      diag->min_T = minT;
      diag->min_phi = minphi;
      diag->R_diag_ratio = rdr;
      /* 1-norm condition of What from its explicit inverse */
      double *Wi = (double *)malloc(sizeof(double) * r * r);
      double *I_r = (double *)calloc(r * r, sizeof(double));
      for (int i = 0; i < r; i++) I_r[i + r * i] = 1.0;
      oracle_lu_solve(r, What, r, I_r, Wi);
      double n1 = 0, n2 = 0;
      for (int j = 0; j < r; j++) {
        double a = 0, b = 0;
        for (int i = 0; i < r; i++) { a += fabs(What[i + r * j]); b += fabs(Wi[i + r * j]); }
        if (a > n1) n1 = a;
        if (b > n2) n2 = b;
      }
      diag->What_cond1 = n1 * n2;
      free(Wi); free(I_r);
    }
    if (phi_out) memcpy(phi_out, phin2, sizeof(double) * Nx);
    memcpy(X, Xn, sizeof(double) * Nx * r);
    memcpy(S, Sn, sizeof(double) * r * r);
    memcpy(W, Wn, sizeof(double) * NOm * r);
    memcpy(T, Tn, sizeof(double) * Nx);
    free(phin2);
    free(Tn);
  } else if (diag) {
    diag->iters = iters;
    diag->dsa_iters = dsa_iters;
  }

  free(ox); free(oy); free(oz); free(w); free(phi0); free(sig_s); free(q);
  free(B0); free(D); free(sig_t); free(idx); free(What); free(WLU);
  free(wpiv); free(beta); free(L0); free(Psi); free(Xn); free(R); free(A); free(P);
  free(Lt0); free(L); free(Wn); free(Sn);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Full-rank SN step (the comparison method of Section 5).            */
/* ------------------------------------------------------------------ */

int oracle_sn_step(const oracle_problem *p, double *psi, double *T,
                   double si_tol, int si_max_iter, double *phi_out,
                   double *outflow, double *inflow) {
  int Nx = p->nx * p->ny, NOm = p->n_polar * p->n_azim;
  double inv_cdt = 1.0 / (p->c * p->dt);
  double *ox = (double *)malloc(sizeof(double) * NOm);
  double *oy = (double *)malloc(sizeof(double) * NOm);
  double *oz = (double *)malloc(sizeof(double) * NOm);
  double *w = (double *)malloc(sizeof(double) * NOm);
  oracle_quadrature(p->n_polar, p->n_azim, ox, oy, oz, w);
  double *sig_s = (double *)malloc(sizeof(double) * Nx);
  double *q = (double *)malloc(sizeof(double) * Nx);
  double *B0 = (double *)malloc(sizeof(double) * Nx);
  double *D = (double *)malloc(sizeof(double) * Nx);
  double *sig_t = (double *)malloc(sizeof(double) * Nx);
  double *phi = (double *)calloc(Nx, sizeof(double));
  double *phin = (double *)malloc(sizeof(double) * Nx);
  double *src = (double *)malloc(sizeof(double) * Nx);
  double *psi0 = (double *)malloc(sizeof(double) * Nx * NOm);
  memcpy(psi0, psi, sizeof(double) * Nx * NOm);
  oracle_coefficients(p, T, sig_s, q, B0, D);
  for (int c = 0; c < Nx; c++) sig_t[c] = oracle_sigma_at(p, c, T[c]) + inv_cdt;
  for (int k = 0; k < NOm; k++)
    for (int c = 0; c < Nx; c++) phi[c] += w[k] * psi0[c + (size_t)Nx * k];
  /* inflow per angle and boundary row; reflective edges lag one iteration */
  double *in_x = (double *)malloc(sizeof(double) * NOm * p->ny);
  double *in_y = (double *)malloc(sizeof(double) * NOm * p->nx);
  int iters = 0, converged = 0;
  while (iters < si_max_iter) {
    sn_inflow(p, ox, oy, iters == 0 ? psi0 : psi, in_x, in_y);
    for (int c = 0; c < Nx; c++) phin[c] = 0;
    for (int k = 0; k < NOm; k++) {
      for (int c = 0; c < Nx; c++)
        src[c] = sig_s[c] * phi[c] / (4.0 * ORACLE_PI) + q[c] + inv_cdt * psi0[c + (size_t)Nx * k];
      oracle_sweep_in(p, ox[k], oy[k], sig_t, src, in_x + (size_t)k * p->ny,
                      in_y + (size_t)k * p->nx, psi + (size_t)Nx * k);
      for (int c = 0; c < Nx; c++) phin[c] += w[k] * psi[c + (size_t)Nx * k];
    }
    iters++;
    double dmax = 0, pmax = 0;
    int bad = 0;  /* a non-finite scalar flux: the iteration diverged */
    for (int c = 0; c < Nx; c++) {
      if (!isfinite(phin[c])) bad = 1;
      if (fabs(phin[c] - phi[c]) > dmax) dmax = fabs(phin[c] - phi[c]);
      if (fabs(phin[c]) > pmax) pmax = fabs(phin[c]);
    }
    if (bad) break;
    if (p->dsa) dsa_correct(p, sig_t, sig_s, phi, phin);
    memcpy(phi, phin, sizeof(double) * Nx);
    if (dmax <= si_tol * pmax) { converged = 1; break; }
  }
  for (int c = 0; c < Nx; c++)
    T[c] = T[c] + p->dt * oracle_sigma_at(p, c, T[c]) * (phi[c] - 4.0 * ORACLE_PI * B0[c]) / D[c];
  if (phi_out) memcpy(phi_out, phi, sizeof(double) * Nx);
  if (outflow && inflow) {
    /* outflow from the last sweep; inflow as that sweep took it */
    int nx = p->nx, ny = p->ny;
    double hx = p->lx / nx, hy = p->ly / ny, o = 0, i_ = 0;
    for (int k = 0; k < NOm; k++) {
      const double *pk = psi + (size_t)Nx * k;
      for (int iy = 0; iy < ny; iy++) {
        o += w[k] * fabs(ox[k]) * hy * pk[iy * nx + (ox[k] < 0 ? 0 : nx - 1)];
        i_ += w[k] * fabs(ox[k]) * hy * in_x[(size_t)k * ny + iy];
      }
      for (int ix = 0; ix < nx; ix++) {
        o += w[k] * fabs(oy[k]) * hx * pk[(oy[k] < 0 ? 0 : ny - 1) * nx + ix];
        i_ += w[k] * fabs(oy[k]) * hx * in_y[(size_t)k * nx + ix];
      }
    }
    *outflow = o;
    *inflow = i_;
  }
  free(ox); free(oy); free(oz); free(w); free(sig_s); free(q); free(B0);
  free(D); free(sig_t); free(phi); free(phin); free(src); free(psi0);
  free(in_x); free(in_y);
  return converged ? iters : -2;
}
