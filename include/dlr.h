/*
 * dlr.h -- C ABI of the GB300 SN-like dynamic-low-rank (DLR) solver for gray
 * thermal radiative transfer in two space dimensions.
 *
 * Method: Haut, Loffeld, Einkemmer, Guthrey, Brunner, Schill, "Efficient
 * SN-like and PN-like Dynamic Low Rank methods for Thermal Radiative
 * Transfer", Section 4 (SN-like DLR scheme) and Algorithm 1 (one implicit time
 * step).  The problem statement follows Section 2: Eqs. (TRT psi), (TRT
 * inflow), (TRT T) with the backward-Euler / Newton linearisation of Section
 * 2.2.  The state is the rank-r factorisation psi(x, Om) = sum_ij X_i(x) S_ij
 * W_j(Om) of Eq. (low rank) plus the material temperature T(x).
 *
 * Discretisation (fixed by this library): nx x ny Cartesian cells on
 * [0,lx] x [0,ly], piecewise-constant (DG0) upwind transport; a product
 * angular quadrature of n_polar Gauss-Legendre cosines mu (ascending) times
 * n_azim equispaced azimuths (a + 1/2) 2 pi / n_azim; angle index
 * k = p * n_azim + a.  Cells are indexed c = iy * nx + ix.  B(T) = a c T^4 /
 * (4 pi).  An edge with a non-negative temperature T_b has isotropic inflow
 * B(T_b) for directions entering it; a negative value means vacuum.
 *
 * Memory and ownership.  dlr_create copies every host input it is given; the
 * library owns all device state of a handle (allocated through the caller's
 * allocator callback when one is given, else cudaMalloc) until dlr_destroy.
 * Output buffers always belong to the caller.  "on_device" arguments say
 * whether a caller pointer is device memory (1) or host memory (0).
 *
 * Streams.  All device work of a handle is enqueued on runtime.stream; when
 * it is 0 the handle creates and owns a non-blocking stream (the step is
 * replayed as CUDA graphs, which cannot be captured on the legacy stream).
 * dlr_step and dlr_step_batch return after enqueueing; getters synchronise
 * the stream.
 *
 * Errors.  Every function returning int returns DLR_OK (0) or a negative
 * DLR_E* code and records a message readable with dlr_last_error() (per
 * thread).  A device-side failure (no convergence, singular matrix, timeout
 * of a bounded wait, non-positive temperature) is sticky on the handle: it is
 * reported by the next synchronising call and by every later dlr_step.
 * Nothing crosses the ABI as a C++ exception.  There is no CPU fallback: on a
 * machine without a usable sm_103 GPU, dlr_create fails with DLR_ECUDA.
 */
#ifndef DLR_GB300_H
#define DLR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DLR_OK 0
#define DLR_EINVAL (-1)     /* bad argument or size */
#define DLR_ENOMEM (-2)     /* allocation failed or HBM budget exceeded */
#define DLR_ENOTCONV (-3)   /* source iteration hit si_max_iter */
#define DLR_ESINGULAR (-4)  /* singular collocation or L-step matrix */
#define DLR_ETIMEOUT (-5)   /* a bounded device-side wait ran out */
#define DLR_ENONPOS (-6)    /* temperature became non-positive */
#define DLR_ECUDA (-7)      /* CUDA runtime error */

#define DLR_FP64 0   /* every kernel in FP64 */
#define DLR_MIXED 1  /* FP32 sweeps and projections, FP64 small linear algebra and T */

#define DLR_SEL_QDEIM 0  /* angles = first r pivots of column-pivoted QR of W^T */
#define DLR_SEL_DEIM 1   /* greedy DEIM of Section 4.2 */

/* dlr_problem.method */
#define DLR_METHOD_DLR 0 /* the SN-like DLR step, Algorithm 1 */
#define DLR_METHOD_SN 1  /* the full-rank SN step it approximates (Section 2.2
                            discretised like Algorithm 1 step 4, over all
                            n_polar * n_azim angles with phi = sum_k w_k psi_k) */

/* Problem statement (Section 2.1-2.2, Algorithm 1 inputs). */
typedef struct dlr_problem {
  int32_t nx, ny;        /* cells per side, >= 1 */
  double lx, ly;         /* domain size, > 0 */
  int32_t n_polar;       /* Gauss-Legendre polar cosines, >= 1 */
  int32_t n_azim;        /* azimuths, >= 1 */
  int32_t rank;          /* r0: 1 <= r0 <= min(32, nx*ny, n_polar*n_azim) */
  double dt;             /* time step, > 0 */
  double c;              /* speed of light, > 0 */
  double a_rad;          /* radiation constant, >= 0 */
  const double *sigma;   /* host, nx*ny absorption opacities, >= 0 (copied) */
  const double *rho_cv;  /* host, nx*ny heat capacities rho*c_v, > 0 (copied) */
  const double *T0;      /* host, nx*ny initial temperatures, > 0 (copied) */
  double T_edge[4];      /* inflow temperature per edge: left, right, bottom,
                            top; < 0 = vacuum */
  int32_t precision;     /* DLR_FP64 or DLR_MIXED */
  int32_t selection;     /* DLR_SEL_QDEIM or DLR_SEL_DEIM */
  int32_t augment;       /* 0: Algorithm 1 as printed; 1: augmented step --
                            step 5 factors [Psi, X0] (2r columns), steps 6-8
                            run at rank 2r, and the SVD of the 2r x 2r S is
                            truncated back to rank r before step 9 (the
                            rank-2r rounding of Section 3 carried over to the
                            SN-like step).  Needs 2r <= min(32, nx*ny, NOm),
                            NOm <= 1024 and DLR_SEL_QDEIM */
  double si_tol;         /* source-iteration tolerance; stop when
                            max|phi_new - phi| <= si_tol * max|phi_new|;
                            <= 0 selects 1e-13 (FP64) or 1e-6 (mixed; the
                            FP32 iterates stall at a few 1e-7 of max|phi|) */
  int32_t si_max_iter;   /* iteration cap (<= 0 selects 1000) */
  int32_t si_fixed_iters;/* > 0: run exactly this many iterations (testing) */
  int32_t allow_nonpositive; /* 0: a non-positive temperature is the sticky
                                error DLR_ENONPOS; 1: it is only counted
                                (dlr_stats.nonpositive_cells).  Algorithm 1
                                does not preserve positivity: a low-rank psi
                                can turn negative ahead of a steep front */
  int32_t method;        /* DLR_METHOD_DLR (rank, selection used) or
                            DLR_METHOD_SN (rank and selection ignored; the
                            state is psi at every cell and angle, starting
                            from the isotropic equilibrium psi = B(T0)) */
  double sigma_texp;     /* temperature-dependent materials, taken at the */
  double cv_texp;        /* step's T0 (Eq. T backward Euler; explicit):    */
  double T_ref;          /* sigma(T) = sigma (T/T_ref)^-sigma_texp and
                            rho c_v(T) = rho_cv (T/T_ref)^cv_texp; exponents
                            0 = constant materials; T_ref <= 0 means 1 */
  int32_t dsa;           /* 1: diffusion synthetic acceleration of the source
                            iteration (Section 4.5): after each round of
                            sweeps the scalar flux is corrected by delta,
                            A delta = M_s (phi^{l+1/2} - phi^l), with A the
                            consistent DG0 diffusion operator (the face
                            penalty (1/8 pi) sum_k w_k |Om_k . n|), solved by
                            Jacobi-preconditioned CG.  The converged step is
                            the same; only the iteration count changes.  The
                            stopping test (si_tol) still measures each round
                            of sweeps' change of phi.  Either method; 0 = off */
  double dsa_tol;        /* CG stop: ||r||_2 <= dsa_tol ||b||_2 (<= 0: 0.1;
                            must be < 1) */
  int32_t dsa_max_iter;  /* CG iteration cap per solve (<= 0: 3); reaching
                            it is not an error (the correction only
                            accelerates the iteration, and a few CG
                            iterations already remove most source
                            iterations) */
  int32_t reflect[4];    /* reflective edges, left, right, bottom, top (1 =
                            reflective; T_edge of that edge is ignored).  A
                            direction entering a reflective edge takes, row by
                            row, the boundary value of its mirror direction
                            (normal component negated; Section 2.1's general
                            boundary conditions).  SN: from the previous
                            source iteration.  DLR: in step 4 the mirror
                            value interpolated through the chosen angles,
                            W0(Om_R) What^-1 Psi, from the previous source
                            iteration; in step 7 the L-step's own boundary
                            values, by a fixed point (at most 5000 passes,
                            else DLR_ENOTCONV).  Not with augment = 1; a
                            reflective left or right edge needs n_azim even
                            (the quadrature's mirror map) */
  int32_t sweep_mode;    /* source-iteration kernel of mixed-precision DLR
                            steps (Algorithm 1 step 4).  The grouped kernel
                            sweeps 2 chosen angles of one quadrant per warp,
                            sums the scalar flux from per-group partials,
                            writes psi once, by a last sweep after the
                            iteration stops, and runs as a loop inside the
                            step's CUDA graph; it serves problems without
                            DSA, reflective edges or the augmented step, and
                            a batch only when all its instances qualify.
                            The per-angle kernel sweeps one angle per warp
                            (every other case).  0 = chosen by dlr_autotune
                            (untuned: grouped for meshes of 2^19 cells or
                            more); 1 = per-angle; 2 = grouped where the
                            problem qualifies.  Both give the same step to
                            FP32 rounding */
  int32_t element;       /* spatial elements (Section 4.4).  0 = piecewise
                            constant (DG0) cells; 1 = bilinear (Q1) upwind
                            DG with the Legendre basis 1, xi, eta, xi eta per
                            cell: psi, X and phi then have 4 coefficients per
                            cell (X is 4 nx ny x r, row 4 c + m, orthonormal
                            in the Q1 L2 inner product), T and the materials
                            stay per cell and the temperature update takes
                            the cell average.  Q1 needs precision = DLR_FP64,
                            the pivoted-QR angle choice, and neither DSA,
                            reflective edges nor the augmented step */
} dlr_problem;

/* Device memory and stream supplied by the caller (e.g. PyTorch). */
typedef struct dlr_runtime {
  void *stream;                                 /* cudaStream_t, 0 = own stream */
  void *(*alloc)(size_t bytes, void *ctx);      /* NULL: cudaMalloc */
  void (*free)(void *ptr, void *ctx);           /* NULL: cudaFree */
  void *ctx;                                    /* passed to alloc / free */
  size_t hbm_budget;  /* if > 0: dlr_create fails with DLR_ENOMEM when the
                         handle's footprint exceeds it */
} dlr_runtime;

typedef struct dlr_handle dlr_handle;

/* Statistics of a handle (all counters since creation). */
typedef struct dlr_stats {
  int64_t steps;             /* completed time steps */
  int64_t si_iters_total;    /* source iterations over all steps */
  int64_t cell_angle_updates;/* sum over steps of nx*ny*r*iterations */
  int32_t si_iters_last;     /* iterations of the last step */
  int32_t status;            /* sticky device status (DLR_OK or DLR_E*) */
  double ms_si_total;        /* device time of the source-iteration kernel,
                                when timing is enabled (else 0) */
  double ms_step_total;      /* device time of whole steps when timing is on */
  int64_t si_launches;       /* timed source-iteration launches */
  int64_t kernel_launches;   /* kernels this handle's steps launched */
  int64_t nonpositive_cells; /* cells with T <= 0 after the last step */
  int64_t dsa_iters_total;   /* CG iterations of all DSA solves (dsa = 1) */
  int32_t sweep_grouped;     /* 1: the last step's source iteration swept two
                                angles of one quadrant per warp (the grouped
                                kernel, see sweep_mode); 0: one per warp */
  int32_t refl_passes_last;  /* fixed-point passes of the last step's L-step
                                with reflective edges (DLR; else 0) */
} dlr_stats;

/* Creates a solver: validates sizes, builds the quadrature and the initial
 * rank-r factors of psi0(x, Om) = B(T0(x)) (X0 = B(T0) then cosine modes,
 * W0 = Om_x^a Om_y^b monomials then Om_z times them, both orthonormalised,
 * S0 = diag(s0, 0, ...)), copies sigma, rho_cv and T0 to the device.  On
 * success *out owns the device state.  Returns DLR_EINVAL, DLR_ENOMEM or
 * DLR_ECUDA on failure (then *out is NULL). */
int dlr_create(const dlr_problem *problem, const dlr_runtime *runtime,
               dlr_handle **out);

/* Enqueues nsteps implicit time steps (Algorithm 1, steps 1-9) on the
 * handle's stream; asynchronous.  Returns a sticky error if an earlier step
 * failed on the device. */
int dlr_step(dlr_handle *h, int32_t nsteps);

/* Enqueues nsteps steps of n independent handles as one batch: each kernel
 * launch covers all handles (one persistent source-iteration launch per step
 * for all of them).  All handles must share precision, selection and the
 * stream of hs[0].  Results equal those of dlr_step on each handle alone. */
int dlr_step_batch(dlr_handle *const *hs, int32_t n, int32_t nsteps);

/* Autotuner of the sweep work plan of a batch (the same handles, in the same
 * order, as later dlr_step_batch calls; n = 1 for dlr_step).  The sweeps of
 * Algorithm 1 step 4 run as units of consecutive 32-row bands of one angle
 * (the per-angle kernel) or of one group of two angles of a quadrant (the
 * grouped kernel, for batches that qualify: see sweep_mode), one CTA per
 * unit; an angle split over several units hands its band edges from unit to
 * unit through global memory.  Candidate plans -- the two kernels, each with
 * no split and with splitting thresholds 2, 1 and 0.5 (an instance's units
 * are halved while the longest is longer than threshold x the average load
 * of one resident CTA) -- are timed on the device, each as reps
 * source-iteration launches of exactly iters iterations on the state the
 * next step starts from (iters near a step's own count: a launch's fixed
 * cost, such as the grouped kernel's last sweep, then weighs as in a step),
 * and the fastest is kept for this handle set and
 * for later batches of the same shape (sorted nx, ny, r, precision).
 * Nothing the next step reads is changed.  *chosen (may be NULL) receives
 * the chosen threshold (0 = no split; dlr_stats.sweep_grouped tells the
 * kernel after the next step); ms (NULL or DLR_AUTOTUNE_CANDIDATES entries)
 * the milliseconds per launch of each candidate: the four thresholds above
 * with the per-angle kernel, then with the grouped one (-1 where the batch
 * cannot take it).  Synchronises.  Without tuning, a batch uses threshold 1
 * and the grouped kernel when it qualifies and its largest mesh has at
 * least 2^19 cells. */
#define DLR_AUTOTUNE_CANDIDATES 8
int dlr_autotune(dlr_handle *const *hs, int32_t n, int32_t iters, int32_t reps,
                 double *chosen, double *ms);

/* Sets the splitting threshold of the sweep work plan of a batch (as in
 * dlr_autotune; 0 = one unit per angle) without timing.  Results do not
 * depend on the plan.  Synchronises.  DLR_EINVAL unless 0 <= split <= 1e9. */
int dlr_set_split(dlr_handle *const *hs, int32_t n, double split);

/* Testing aid for failure detection (no paper counterpart): gives the batch
 * of these handles its finest sweep work plan, with one unit whose bands
 * wait for the top row of the band below it in another CTA pointed at an
 * edge row that nothing writes.  The next step's wait for that row gives up
 * after its time bound (4 s), every instance of the batch reports the sticky
 * DLR_ETIMEOUT, and the GPU context stays usable (nothing faults or hangs).
 * DLR_EINVAL if no angle spans more than one unit (ny <= 32 x sweep warps).
 * Synchronises. */
int dlr_debug_lose_edge(dlr_handle *const *hs, int32_t n);

/* Testing aid (no paper counterpart): the fifth-generation tensor-core
 * contraction of the mixed-precision projections of Algorithm 1 steps 6
 * and 7 (tcgen05 MMAs of kind TF32 with the operands in shared memory and
 * the FP32 accumulator in tensor memory; each operand split into two TF32
 * parts and a product summed as hi lo + lo hi + hi hi) on plain device
 * arrays:
 * D (m x n, row-major FP32) = A (m x k, row-major) times B^T (B: n x k,
 * row-major), with m in {128, 256}, n in {16, 32}, k a multiple of 32, A
 * and B 16-byte aligned (DLR_EINVAL otherwise).  All pointers are device
 * memory owned by the caller.  One CTA on stream; synchronises.  Returns
 * DLR_OK, DLR_ETIMEOUT if a completion wait ran out (1 s), or DLR_ECUDA. */
int dlr_debug_tc_gemm(const float *A, const float *B, int32_t m, int32_t n, int32_t k, float *D,
                      void *stream);

/* Copies the material temperature T (Section 2.1, the T of Eq. (temperature
 * update) after the last step; nx*ny FP64, cell c = iy nx + ix) into out;
 * synchronises.  Returns the sticky device status if a step failed. */
int dlr_get_T(dlr_handle *h, double *out, int32_t out_on_device);

/* Replaces the temperature T (Section 2.1; nx*ny FP64) with in: the T0 of
 * the next step's linearisation (Section 2.2).  Enqueued on the stream.  A
 * pageable host buffer is consumed before return; a pinned one must stay
 * unchanged until the stream has executed the copy. */
int dlr_set_T(dlr_handle *h, const double *in, int32_t in_on_device);

/* Copies the low-rank factors of psi = X S W^T (Section 4: the rank-r
 * representation Algorithm 1 advances; W in the quadrature's discrete inner
 * product): X (rows x r, column-major, hx*hy*X^T X = I; rows = nx*ny, or
 * 4*nx*ny plain Legendre coefficients with element = 1), S (r x r,
 * column-major), W (NOm x r, column-major, sum_k w_k W_ki W_kj = d_ij), all
 * FP64 (X is widened in mixed precision); rotated to the SVD basis of S
 * first when the step keeps S general.  *r_out = r.  Any pointer may be NULL.
 * Synchronises; DLR_EINVAL for a full-rank SN handle. */
int dlr_get_factors(dlr_handle *h, double *X, double *S, double *W,
                    int32_t *r_out, int32_t out_on_device);

/* Replaces the factors (same layouts as dlr_get_factors): the X0, S0, W0 the
 * next step of Algorithm 1 starts from.  Used to start from a given state.
 * DLR_EINVAL for a full-rank SN handle. */
int dlr_set_factors(dlr_handle *h, const double *X, const double *S,
                    const double *W, int32_t in_on_device);

/* Copies the angular quadrature of the discrete ordinates (Section 2.2; the
 * product rule of Gauss-Legendre polar cosines and equispaced azimuths):
 * omega_xyz (NOm x 3 row-major: Om_x, Om_y, Om_z of angle k = p n_azim + a)
 * and weights w (NOm, summing to 4 pi).  Either may be NULL. */
int dlr_get_quadrature(dlr_handle *h, double *omega_xyz, double *w);

/* The r angle indices chosen in the last step (Algorithm 1 step 2), or -1
 * before the first step.  Synchronises. */
int dlr_get_selected(dlr_handle *h, int32_t *idx);

/* The angular flux psi (rows x NOm, column-major: psi[c + rows*k] for row c
 * and angle k of dlr_get_quadrature, FP64; rows = nx*ny, or 4*nx*ny plain
 * Legendre coefficients with element = 1).  dlr_get_psi copies the state of
 * a full-rank SN handle (widened from FP32 in mixed precision), or forms
 * psi = X S W^T of a DLR handle on the device (Section 4: the low-rank
 * form; like dlr_get_factors it first rotates the factors to the SVD basis
 * of S; a host destination goes through a temporary device array of the
 * same size); it synchronises.  dlr_set_psi replaces the state of a
 * full-rank SN handle (DLR_EINVAL for a DLR handle: dlr_set_factors); it is
 * enqueued (a pageable host buffer is consumed before return). */
int dlr_get_psi(dlr_handle *h, double *out, int32_t out_on_device);
int dlr_set_psi(dlr_handle *h, const double *in, int32_t in_on_device);

/* Statistics; synchronises. */
int dlr_get_stats(dlr_handle *h, dlr_stats *out);

/* Enables (1) or disables (0) CUDA-event timing of the source-iteration
 * kernel and of whole steps (read back through dlr_get_stats). */
int dlr_set_timing(dlr_handle *h, int32_t enable);

/* Sets the isotropic inflow value psi_iso (>= 0, a value of psi, not a
 * temperature) of one edge (0 left, 1 right, 2 bottom, 3 top) for the
 * following steps. */
int dlr_set_edge_inflow(dlr_handle *h, int32_t edge, double psi_iso);

/* Device bytes a handle for this problem would hold (no allocation). */
size_t dlr_footprint_bytes(const dlr_problem *problem);

/* Releases the handle and its device state (synchronises its stream). */
void dlr_destroy(dlr_handle *h);

/* Message of the last error on this thread ("" if none). */
const char *dlr_last_error(void);

/* Hot-kernel entry point (the DG0 upwind sweep of Section 4.4 used by
 * Algorithm 1 step 4), for testing the sweep alone.  For each of n_dir
 * directions d with in-plane components dirs[2d], dirs[2d+1] (host), solves
 *   |ox|/hx (psi_c - psi_west) + |oy|/hy (psi_c - psi_south) + sigma_t,c psi_c
 *     = src[d*N + c]
 * in upwind order, with edge inflow psi_edge[4] (host; left, right, bottom,
 * top).  sigma_t (N), src (n_dir*N) and psi (n_dir*N, output) are device
 * arrays of double (precision DLR_FP64) or float (DLR_MIXED), N = nx*ny.
 * Synchronous on stream.  Returns DLR_EINVAL, DLR_ETIMEOUT or DLR_ECUDA on
 * failure. */
int dlr_sweep(int32_t nx, int32_t ny, double lx, double ly, int32_t n_dir,
              const double *dirs, const double *psi_edge, int32_t precision,
              const void *sigma_t, const void *src, void *psi, void *stream);

/* Allocation-free variant of dlr_sweep.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, for
 * example an application whose device memory is entirely held by another
 * allocator (a framework's caching allocator that reserved the pool, so a
 * fresh cudaMalloc fails or fragments it), or a latency-critical loop in
 * which cudaMalloc / cudaFree, which may synchronise the device, are not
 * allowed.  dlr_sweep allocates its small scratch (the directions, the edge
 * inflow values and a wait flag) stream-ordered on every call; this variant
 * keeps that scratch in one fixed array compiled into the library instead
 * (about 64 KB, held on every GPU that loads the library until the process
 * exits) and calls no allocating routine.
 *
 * Arguments, layouts and results are those of dlr_sweep; inputs and outputs
 * stay the caller's.  n_dir may not exceed DLR_SWEEP_NOALLOC_MAX_DIRS
 * (DLR_EINVAL otherwise), and the mesh-width limit of dlr_sweep applies
 * (DLR_EINVAL).  Every call looks up the array's device address on the
 * device current at the call (no cached address can go stale after a
 * context teardown); the first lookup on a device may load the library's
 * device code there, so make the first call before any stream capture.  All calls share the one array,
 * which keeps the last call's contents (the wait flag is cleared on every
 * call): calls that overlap on the GPU, from several streams or threads at
 * once, race on it and must be serialised by the caller.  Synchronous on
 * stream.  Returns DLR_OK, DLR_EINVAL, DLR_ETIMEOUT or DLR_ECUDA. */
#define DLR_SWEEP_NOALLOC_MAX_DIRS 4096
int dlr_sweep_noalloc(int32_t nx, int32_t ny, double lx, double ly, int32_t n_dir,
                      const double *dirs, const double *psi_edge, int32_t precision,
                      const void *sigma_t, const void *src, void *psi, void *stream);

#ifdef __cplusplus
}
#endif
#endif
