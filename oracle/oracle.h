/*
 * oracle.h -- plain FP64 CPU reference of the SN-like dynamic-low-rank (DLR)
 * time step for gray thermal radiative transfer in 2-D (Haut et al.,
 * "Efficient SN-like and PN-like Dynamic Low Rank methods for Thermal
 * Radiative Transfer", Section 4 and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * path.
 *
 * Conventions (all arrays FP64, caller-owned):
 *   cells      c = iy*nx + ix, cell centres ((ix+1/2)hx, (iy+1/2)hy)
 *   angles     k = p*n_azim + a  (Gauss-Legendre polar index p, azimuth a)
 *   matrices   column-major: X[c + Nx*i] (Nx x r), W[k + NOm*j] (NOm x r),
 *              S[i + r*j] (r x r), L[i + r*k] (r x NOm)
 *   edges      0 = left (x=0), 1 = right (x=lx), 2 = bottom (y=0), 3 = top
 *   orthonormality  hx*hy*sum_c X_ci X_cj = delta_ij,
 *                   sum_k w_k W_ki W_kj = delta_ij
 */
#ifndef DLR_ORACLE_H
#define DLR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny;          /* cells */
  double lx, ly;       /* domain [0,lx] x [0,ly] */
  int n_polar, n_azim; /* product quadrature, NOm = n_polar*n_azim */
  double dt, c, a_rad; /* time step, speed of light, radiation constant */
  const double *sigma;  /* Nx absorption opacity */
  const double *rho_cv; /* Nx heat capacity */
  double psi_edge[4];  /* isotropic inflow value of psi per edge; 0 = vacuum */
  /* temperature dependence (reading R16): sigma(T) = sigma (T/T_ref)^-sigma_texp,
   * rho c_v(T) = rho_cv (T/T_ref)^cv_texp, both taken at the step's T0
   * (explicit, Eq. T backward Euler); exponents 0 = constant; T_ref <= 0
   * means 1 */
  double sigma_texp, cv_texp, T_ref;
  /* diffusion synthetic acceleration of the source iteration (Section 4.5,
   * reading R17): dsa = 1 turns it on; the CG solve of each DSA step stops
   * at ||r||_2 <= dsa_tol ||b||_2 or after dsa_max_iter iterations */
  int dsa;
  double dsa_tol;
  int dsa_max_iter;
  /* reflective edges (left, right, bottom, top; reading R18, full-rank SN
   * only): 1 = the edge mirrors the angular flux, 0 = psi_edge inflow */
  int reflect[4];
} oracle_problem;

typedef struct {
  int selection;          /* 0 = pivoted-QR (Q-DEIM) angle choice, 1 = DEIM */
  const int *forced_idx;  /* if non-NULL: use these r angle indices */
  double si_tol;          /* relative sup-norm stopping tolerance */
  int si_max_iter;        /* iteration cap (returns -2 if reached) */
  int si_fixed_iters;     /* > 0: run exactly this many iterations */
  int canonicalize;       /* 1: rotate factors to the SVD of S */
  int augment;            /* 1: augmented step (reading R15): steps 5-8 on
                             orth([Psi, X0]) at rank 2r, then the SVD of the
                             2r x 2r S truncated back to rank r */
} oracle_dlr_opts;

typedef struct {
  int iters;              /* source iterations taken */
  int dsa_iters;          /* CG iterations of all DSA solves of the step */
  double E_before, E_after;  /* sum_c h^2 (rho_cv T + phi/c) */
  double outflow, inflow;    /* boundary energy rates of the new psi */
  double residual;        /* E_after - E_before + dt (outflow - inflow) */
  double min_T, min_phi;
  double What_cond1;      /* 1-norm condition estimate of What (explicit inverse) */
  double R_diag_ratio;    /* min_j |R_jj| / max_j |R_jj| of the Psi = X R factor */
} oracle_dlr_diag;

/* Planck function B(T) = a c T^4 / (4 pi) (reading of the undefined B). */
/* Threads of the OpenMP loops (n <= 0: all processors); results do not
 * depend on the count.  Without OpenMP the oracle runs on one thread. */
void oracle_set_threads(int n);
int oracle_get_threads(void);

double oracle_planck(double a_rad, double c, double T);

/* sigma(T0) and rho c_v(T0) of cell c (reading R16). */
double oracle_sigma_at(const oracle_problem *p, int c, double T0);
double oracle_rhocv_at(const oracle_problem *p, int c, double T0);

/* Product quadrature: Gauss-Legendre mu ascending x equispaced azimuths. */
void oracle_quadrature(int n_polar, int n_azim, double *ox, double *oy,
                       double *oz, double *w);

/* Linearised coefficients of Section 2.2 (reading R1): sigma_s, q, B0, D. */
void oracle_coefficients(const oracle_problem *p, const double *T0,
                         double *sigma_s, double *q, double *B0, double *D);

/* One DG0 upwind transport sweep in direction (ox, oy):
 * (ox d/dx + oy d/dy + sigma_t) psi = src, with the problem's edge inflow. */
void oracle_sweep(const oracle_problem *p, double ox, double oy,
                  const double *sigma_t, const double *src, double *psi);

/* DSA (Section 4.5, reading R17): the penalty coefficient of faces normal
 * to x (axis 0) or y (axis 1); out = A u for the DG0 diffusion operator
 * A = (1/3) sum_j Fbar_j^T M_t^{-1} Fbar_j + F0 + M_a; its diagonal; and
 * Jacobi-preconditioned CG for A x = b (returns the iterations). */
double oracle_dsa_kappa(int n_polar, int n_azim, int axis);
void oracle_dsa_apply(const oracle_problem *p, const double *sig_t,
                      const double *sig_a, const double *u, double *out);
void oracle_dsa_diag(const oracle_problem *p, const double *sig_t,
                     const double *sig_a, double *d);
int oracle_dsa_solve(const oracle_problem *p, const double *sig_t,
                     const double *sig_a, const double *b, double tol,
                     int max_iter, double *x);

/* The sweep with an inflow value per boundary row and column:
 * in_x[iy] enters the upwind x-face of row iy, in_y[ix] the upwind y-face of
 * column ix. */
void oracle_sweep_in(const oracle_problem *p, double ox, double oy,
                     const double *sigma_t, const double *src,
                     const double *in_x, const double *in_y, double *psi);

/* Bilinear (Q1) upwind DG sweep of Section 4.4 in direction (ox, oy): per
 * cell the coefficients of 1, xi, eta, xi eta (reference coordinates of the
 * cell), 4 per cell in src and psi; in_x[2 iy + m] and in_y[2 ix + m] the
 * inflow through the upwind x-face of row iy and y-face of column ix as
 * constant (m = 0) and slope (m = 1) along the face. */
void oracle_sweep_q1(const oracle_problem *p, double ox, double oy,
                     const double *sigma_t, const double *src,
                     const double *in_x, const double *in_y, double *psi);

/* Full-rank SN step on Q1 elements: psi[4 (k Nx + c) + m] (coefficients of
 * 1, xi, eta, xi eta), T per cell, phi_out 4 Nx; the temperature update uses
 * the cell average of phi.  Returns iterations, or -2 at the cap. */
int oracle_sn_step_q1(const oracle_problem *p, double *psi, double *T,
                      double si_tol, int si_max_iter, double *phi_out,
                      double *outflow, double *inflow);

/* One SN-like DLR step (Algorithm 1) on Q1 elements: X (4 Nx x r) holds Q1
 * coefficients per cell, orthonormal in the L2 inner product of Q1 fields;
 * S (r x r), W (NOm x r), T (Nx) as for DG0.  Pivoted-QR angle choice, no
 * canonical rotation.  Returns 0, -1 or -2 (SI cap). */
int oracle_dlr_step_q1(const oracle_problem *p, int r, double *X, double *S, double *W,
                       double *T, double si_tol, int si_max_iter, int *iters_out,
                       double *phi_out);

/* DSA on Q1 elements (reading R20), dense (4 Nx x 4 Nx, column major): the
 * DG derivative D_j (axis 0: x, 1: y) and the operator
 * A = (1/3) sum_j D_j^T M_t^{-1} D_j + F0 + M_a. */
void oracle_q1_deriv(const oracle_problem *p, int axis, double *Dm);
void oracle_dsa_matrix_q1(const oracle_problem *p, const double *sig_t, const double *sig_a,
                          double *A);

/* Index of the mirror image of quadrature angle k (axis 0: x component
 * negated, needs n_azim even; axis 1: y component negated), reading R18. */
int oracle_reflect_index(int n_polar, int n_azim, int k, int axis);

/* Dense linear algebra building blocks. */
int oracle_lu_solve(int n, const double *A, int nrhs, const double *B,
                    double *Xout);
void oracle_householder_qr(int m, int n, const double *A, double *Q,
                           double *R);
int oracle_jacobi_svd(int n, const double *A, double *U, double *s,
                      double *V);
int oracle_qdeim(int n, int r, const double *W, int *idx);
int oracle_deim(int n, int r, const double *W, int *idx);

/* Deterministic rank-r initial factors for psi0(x, Om) = B(T0(x)). */
int oracle_initial_factors(const oracle_problem *p, const double *T0, int r,
                           double *X0, double *S0, double *W0);

/* L-step of Algorithm 1 step 7 for given X (new space basis), coefficient
 * fields and projected old state Lt0 (r x NOm).  Writes L (r x NOm). */
int oracle_lstep(const oracle_problem *p, int r, const double *X,
                 const double *sigma_t, const double *sigma_s,
                 const double *q, const double *Lt0, double *L);
/* The same with an extra inflow vector per angle added to Q_k, gext
 * (r x NOm, NULL: none); a reflective edge adds no constant inflow. */
int oracle_lstep_g(const oracle_problem *p, int r, const double *X,
                   const double *sigma_t, const double *sigma_s,
                   const double *q, const double *Lt0, const double *gext, double *L);

/* Steps 1-4 of Algorithm 1 at the given angle indices: coefficients from
 * T0, psi0 at the chosen angles, source iteration of the collocation system.
 * Writes Psi (Nx x r); returns 0, -1 (singular What), -2 (SI cap). */
int oracle_collocation(const oracle_problem *p, int r, const double *X0,
                       const double *S0, const double *W0, const double *T0,
                       const int *idx, double tol, int max_iter, int fixed,
                       double *Psi, int *iters);

/* One SN-like DLR step (Algorithm 1).  X (Nx x r), S (r x r), W (NOm x r)
 * and T (Nx) are read as the state at t0 and overwritten with the state at
 * t0 + dt.  idx_out (r), phi_out (Nx) and diag may be NULL.
 * Returns 0, -1 on bad input / singular matrix, -2 if SI hit its cap. */
int oracle_dlr_step(const oracle_problem *p, int r, double *X, double *S,
                    double *W, double *T, const oracle_dlr_opts *opt,
                    int *idx_out, double *phi_out, oracle_dlr_diag *diag);

/* One full-rank SN step with source iteration.  psi (Nx x NOm, column k is
 * angle k) and T are overwritten.  Returns iterations, or -2 at the cap. */
int oracle_sn_step(const oracle_problem *p, double *psi, double *T,
                   double si_tol, int si_max_iter, double *phi_out,
                   double *outflow, double *inflow);

#ifdef __cplusplus
}
#endif
#endif
