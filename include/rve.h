/*
 * rve.h -- C ABI of the GB300 ringing-free FFT homogenisation solver.
 *
 * The library solves the small-strain periodic cell (RVE) problem of
 * "Non-convex, ringing-free, FFT-accelerated solver using an incremental
 * approximate energy functional" (arXiv 2207.10657):
 *
 *   find the strain field eps = E + eps~ (Sec. 2, Eq. (1)) such that
 *   G : sigma(eps) = 0 (Eq. (6)), with G the compatibility projection built
 *   from the linear finite-element (ringing-free) gradient (Sec. 2.1,
 *   Eq. (9)), sigma the isotropic damage law of Appendix A, solved by the
 *   trust-region Newton-CG method of Algorithm 2 whose ratio test uses the
 *   first-order incremental energy (Sec. 2.2.1, Eqs. (18)-(19)) and whose
 *   sub-problem is Steihaug CG (Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: dims[0] = Nx, dims[1] = Ny, dims[2] = Nz (ignored for ndim = 2),
 *    unit voxels, periodic.  Nvox = Nx*Ny(*Nz).  Every dim must be even,
 *    >= 2, <= 1024 and have no prime factor other than 2, 3 and 5.
 *  - Fields are structure-of-arrays, component-major: element (c, z, y, x)
 *    at offset ((c*Nz + z)*Ny + y)*Nx + x, x fastest.  Components are
 *    Mandel-orthonormal: 3D (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12),
 *    2D plane strain (11, 22, sqrt2*12).  ncomp = 6 (3D) or 3 (2D).  With
 *    the simplex element (rve_solver_opts.element = 1) a field has nq
 *    strain points per voxel (nq = 2 triangles in 2D, 6 tetrahedra in
 *    3D): ncomp x nq x Nvox, element (c, q, [z,] y, x) at
 *    (((c*nq + q)*Nz + z)*Ny + y)*Nx + x, and per-point scalar fields
 *    nq x Nvox.
 *  - Real type: float when the context was created with precision 32,
 *    double with precision 64.  Pointers named *_dev are DEVICE pointers,
 *    owned by the caller, 16-byte aligned, read/written on the context's
 *    stream; the call returns before the device work completes unless it
 *    returns scalars to the host (those calls synchronise the stream).
 *  - Pointers named *_host are host pointers (pinned or pageable).
 *  - Errors: every call returns an rve_status; nothing aborts, traps or
 *    throws.  rve_last_error() gives a message for the last failure.
 *  - Reductions (energies, CG scalars, the trust-region ratio) are FP64 on
 *    the device whatever the field precision.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rve_ctx* rve_t; /* opaque; owned by the library */

typedef enum {
  RVE_OK = 0,
  RVE_ERR_ARG = -1,           /* invalid argument (size, pointer, option) */
  RVE_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  RVE_ERR_OOM = -3,           /* device allocation failed */
  RVE_ERR_NOT_CONVERGED = -4, /* iteration caps reached */
  RVE_ERR_NONFINITE = -5,     /* NaN/Inf met in a reduction */
  RVE_ERR_TIMEOUT = -6        /* a bounded device wait gave up: the x-forward
                                 pass of 3D FP32 grids waits on an mbarrier
                                 for its bulk tensor copies (at most about a
                                 second); the calls that read the device
                                 scalars back (solve steps, Steihaug, dot
                                 products) report it.  Every device wait of the
                                 library is bounded. */
} rve_status;

/* One material phase, indexed by the phase id stored per voxel.
 * Isotropic elasticity (E, nu); if damaging != 0, isotropic damage
 * E -> (1-D) E (Eq. (22)) driven by the tension strain measure
 * kappa = |eps^(t)| (Eq. (A.1)), bilinear law (Eq. (A.3)) read as
 * D = kappaf (kappa - kappa0) / (kappa (kappaf - kappa0)) on
 * (kappa0, kappaf), 0 below, 1 from kappaf on. */
typedef struct {
  double E, nu;
  int damaging;
  double kappa0, kappaf;
} rve_phase;

/* Solver options (Algorithm 2 hyper-parameters; the paper gives no values). */
typedef struct {
  double eta_eq;      /* converged when |G:sigma| / |sigma| <= eta_eq */
  double eta_nr;      /* ... or |d_eps| / |eps| <= eta_nr (0 disables) */
  double eta_cg;      /* relative Steihaug-CG tolerance |r| <= eta_cg |g| */
  double eta_up;      /* accept a trial step when rho_bar > eta_up */
  double R0, Rmax;    /* initial / maximum trust radius (unnormalised norm) */
  int max_nr, max_cg; /* Newton and CG iteration caps */
  double restart_thr; /* Powell restart threshold, Eq. (20): 0.2 */
  int precision;      /* 32 (FP32 fields) or 64 (FP64 fields) */
  int hessian;        /* 0: secant (1-D) C (default); 1: symmetric part of the
                         consistent damage tangent, (1-D) C - D'(kappa)/2
                         ((C:eps) (x) n + n (x) (C:eps)) with n = eps^(t)/kappa
                         on loading voxels (Appendix A; kappa^2 is a spectral
                         function of eps, so d kappa/d eps = n).  Used by the
                         Hessian-vector products and the model change of the
                         trust-region step; costs 4 B/voxel per product plus
                         C:eps and n on loading voxels, and 13 reals per voxel
                         of storage.  The batched solver (rve_batch_create)
                         takes 0 or 1 as well; with 1 it prepares the per-voxel
                         data once per member and accepted state, and every
                         batched tangent product (rve_batch_hessp too) uses
                         the state's consistent tangent. */
  int passes;         /* 0: FP32 fields use the passes compiled for the axis
                         lengths 32, 64, 128, 256, 512, 96, 192 and 384
                         (per axis), with the Steihaug-CG iterate / residual
                         update fused into the x-inverse pass where Nx is
                         one of them (default);
                         1: the generic runtime passes only, with separate
                         CG update kernels (the same method through a second
                         implementation, for cross-checks); 2: the compiled
                         passes with the CG scalars and updates of the
                         generic path (d.Hd from the stored product, separate
                         update kernels); 3: as 0, and on 3D grids with
                         Nx = Ny in {64, 96, 128, 192, 256} the x and y
                         transforms of each direction in one pass (clusters
                         of four CTAs sharing a z-plane's component through
                         distributed shared memory; three passes per
                         product, correct but slower than the five of 0 on
                         this hardware).  FP64 fields and other lengths
                         always use the generic passes. */
  int element;        /* finite-element gradient the projection is built from
                         (Sec. 2.1, Eq. (9)): 0: one bilinear / trilinear
                         element per voxel, one quadrature point (default);
                         1: linear simplices, every voxel split along its
                         main diagonal into the simplices of the axis
                         permutations (Kuhn), one quadrature point each: in
                         2D the two triangles of axis order (x, y) and (y, x),
                         in 3D the six tetrahedra of the permutations of
                         (x, y, z) in lexicographic order; secant Hessian
                         only.  With 1 every strain-sized field holds
                         ncomp x nq x Nvox reals (nq = 2 or 6), layout
                         [c][q][z][y][x] (q the simplex in the order above),
                         and every per-point scalar field (history, damage)
                         nq x Nvox; the mean strain and stress average over
                         all simplices.  3D runs on the generic passes and
                         takes Nx <= 227 and Nz <= 341 (FP32) / 177 (FP64);
                         rve_create returns RVE_ERR_ARG past that. */
} rve_solver_opts;

/* Per-load-step statistics. */
typedef struct {
  int nr_iters, cg_iters, hv_products, restarts, rejected, boundary_hits;
  int converged;
  double rel_residual; /* |G:sigma| / |sigma| at exit */
  double R;            /* trust radius at exit */
  double mean_stress[6], mean_strain[6];
} rve_step_report;

/* Exit of one Steihaug-CG solve (Algorithm 1), from rve_steihaug. */
typedef struct {
  int status;      /* 1 converged (|r| <= eta_cg |g|), 2 boundary (|z| = R,
                      the non-negative root), 3 negative curvature (d.Hd <= 0:
                      the root of |z + tau d| = R with the lower model value),
                      4 max_cg reached, 5 zero right-hand side (z = 0) */
  int iters;       /* CG iterations (Hessian-vector products of directions) */
  int hv_products; /* products including the restarts of Eq. (20) */
  int restarts;    /* Powell restarts (Eq. (20)) */
} rve_cg_report;

/* Fill opts with defaults: eta_eq 1e-6, eta_nr 0, eta_cg 1e-2, eta_up 0.1,
 * R0 = Rmax = 0 (meaning "10 sqrt(Nvox) |dE|" at the first load step),
 * max_nr 50, max_cg 1000, restart_thr 0.2, precision 32, hessian 0,
 * passes 0, element 0. */
void rve_default_opts(rve_solver_opts* opts);

/* Create a context.  Sec. 2 (cell, strain split), Appendix A (phases).
 *  dims, ndim     grid (see conventions); ndim 2 = plane strain.
 *  phase_ids_dev  Nvox uint8 phase ids (device); copied, may be freed after.
 *  phases_host    nphase entries (1..16), copied.
 *  opts_host      may be NULL for defaults; copied.
 *  stream         cudaStream_t (as void*) all work is issued on; NULL =
 *                 the legacy default stream.
 *  out            receives the handle.
 * Allocates every workspace (spectra, CG vectors, FP64 scalars) up front;
 * fails with RVE_ERR_OOM if the device cannot hold them.  The state starts
 * at eps = 0, kappa_n = 0, all components strain-controlled. */
rve_status rve_create(const int dims[3], int ndim, const uint8_t* phase_ids_dev,
                      const rve_phase* phases_host, int nphase,
                      const rve_solver_opts* opts_host, void* stream, rve_t* out);

/* Set the state: total strain (ncomp x Nvox) and committed history kappa_n
 * (Nvox, NULL = 0), both of the context's real type.  Recomputes sigma and
 * D at the state (Appendix A, with kappa = max(kappa_n, kappa(eps))). */
rve_status rve_set_state(rve_t, const void* strain_dev, const void* kappa_hist_dev);

/* Copy out the state; any pointer may be NULL.  strain_dev / stress_dev:
 * ncomp x Nvox; kappa_dev (committed history) / damage_dev (damage D at the
 * state): Nvox.  All of the context's real type. */
rve_status rve_get_state(rve_t, void* strain_dev, void* kappa_dev, void* stress_dev,
                         void* damage_dev);

/* Replace the frozen damage field used by rve_hessp (Nvox values in [0,1],
 * context's real type).  For the Hessian-vector product on a damage
 * snapshot (benchmarks, tests).  With opts.hessian = 1 the rank-one part of
 * the consistent tangent stays the one of the last evaluated state. */
rve_status rve_set_damage(rve_t, const void* damage_dev);

/* Stress-controlled mean components (zero mean stress): free_mask[c] != 0
 * for Mandel component c.  Sets Ghat(0) = P_free (mixed control, Sec. 3.3). */
rve_status rve_set_free_mask(rve_t, const uint8_t free_mask_host[6]);

/* Per-phase eigenstrain (Algorithm 2: the constitutive law is evaluated at
 * eps_eval = eps + eps_eig; Sec. 3.3 imposes a growing eigenstrain on the
 * pixels holding ASR product under free expansion).  eig_host: host array of
 * nphase x ncomp doubles, phase-major, Mandel order of the fields; nphase
 * must equal the context's phase count.  Copied (the caller keeps
 * ownership).  Every later constitutive evaluation (load steps, the initial
 * state of a step, rve_energy_grad, rve_set_state) adds row p to the strain
 * of the voxels of phase p; the unknown eps, the gradient G:sigma, the
 * Hessian (secant at the damage so evaluated), the mean strain of the step
 * report and the |d eps|/|eps| measure stay those of eps.  The current state
 * (stress, damage, kappa) is re-evaluated at once.  The sign is the paper's:
 * a stress-free expansion e of a phase is eps_eig = -e.  NULL removes the
 * eigenstrain.  RVE_ERR_ARG on a wrong nphase or a non-finite entry. */
rve_status rve_set_eigenstrain(rve_t, const double* eig_host, int nphase);

/* Hessian-vector product of Eq. (8) with the tangent frozen at the state:
 * out = G : ((1 - D) C : v) (secant), or with the symmetric consistent
 * tangent of the state when the context was created with opts.hessian = 1.
 * v_dev, out_dev: ncomp x Nvox real; they may alias.  The product is:
 * tangent (Eq. (13)), forward real FFT, per-frequency projection Ghat(k)
 * from the FE gradient (Eqs. (5), (9)), inverse FFT. */
rve_status rve_hessp(rve_t, const void* v_dev, void* out_dev);

/* Projection alone, out = G : v (Eqs. (4)-(5)).  May alias. */
rve_status rve_project(rve_t, const void* v_dev, void* out_dev);

/* Energy quantities of a trial increment p (ncomp x Nvox, NULL = 0) from
 * the state eps (Sec. 2.2.1, Algorithm 2):
 *   dW_bar = 1/2 (sigma(eps) + sigma(eps + p)) : p        (Eq. (18))
 *   dm     = sigma(eps) : p + 1/2 p : (1-D) C : p           (Delta m)
 *   grad_dev (may be NULL) = G : sigma(eps + p)             (Eq. (12))
 * dW_bar_host / dm_host may be NULL.  Synchronises the stream. */
rve_status rve_energy_grad(rve_t, const void* p_dev, double* dW_bar_host, double* dm_host,
                           void* grad_dev);

/* One load step of Algorithm 2: eps += dE (uniform, strain-controlled
 * components), optionally eps += init_incr (a compatible warm-start
 * fluctuation increment, ncomp x Nvox, NULL = none), then trust-region
 * Newton iterations with Steihaug CG until converged; on convergence
 * kappa_n <- max(kappa_n, kappa(eps)).  free_mask_host may be NULL (keep the
 * current mask).  rep_host may be NULL.  Returns RVE_ERR_NOT_CONVERGED
 * (state kept, history not committed) when max_nr is exhausted. */
rve_status rve_solve_step(rve_t, const double dE_host[6], const uint8_t free_mask_host[6],
                          const void* init_incr_dev, rve_step_report* rep_host);

/* One Steihaug-CG solve (Algorithm 1) at the current state, the
 * sub-problem of one Newton iteration of Algorithm 2: minimise the quadratic
 * model m(z) = g : z + 1/2 z : H z over compatible z with |z| <= R, where
 * g = G : sigma(state) (Eq. (12)) and H the Hessian of Eq. (8) frozen at the
 * state (secant, or the symmetric consistent tangent with opts.hessian = 1).
 * z_0 = 0, r_0 = g, d_0 = -r_0; exits on d.Hd <= 0, on |z| reaching R, on
 * |r| <= eta_cg |g| or after opts.max_cg iterations; Powell restart with
 * opts.restart_thr (Eq. (20)).  Norms are unnormalised sums over every voxel
 * and Mandel entry.
 *  R         trust radius (> 0)
 *  eta_cg    relative CG tolerance, in (0, 1)
 *  z_dev     ncomp x Nvox of the context's real type: receives z
 *  rep_host  may be NULL
 * The state, the trust radius of the load steps and the options are not
 * changed.  Synchronises the stream.  RVE_ERR_ARG on a bad R / eta_cg / NULL
 * z_dev; RVE_ERR_NONFINITE when a CG scalar is not finite. */
rve_status rve_steihaug(rve_t, double R, double eta_cg, void* z_dev, rve_cg_report* rep_host);

/* One load step solved by L-BFGS instead of the trust-region Newton-CG
 * iteration: the quasi-Newton method that the paper notes becomes usable
 * once the first-order incremental energy (Eq. (18)) stands in for the
 * objective (Sec. 2.2.1, after Eq. (20)); no algorithm is printed, so this is
 * Nocedal & Wright's L-BFGS (Alg. 7.5, two-loop recursion Alg. 7.4) on the
 * compatible strain fields with gradient G:sigma and a backtracking Armijo
 * line search on dW_bar: halve s = alpha p (alpha from 1, at most 40 times)
 * until 1/2 (sigma(eps) + sigma(eps + s)) : s <= 1e-4 sigma(eps) : s.  A pair
 * (s, y = G:sigma_new - G:sigma) is kept when s.y > 1e-12 |s||y|; H0 =
 * gamma I with gamma = s.y / y.y of the newest pair, 1 / max_phase(3 lambda
 * + 2 mu) before the first.  A direction that is not a descent direction
 * drops the pairs.  Converged when |G:sigma| / |sigma| <= opts.eta_eq.
 *  dE_host, free_mask_host  as for rve_solve_step (mask may be NULL)
 *  memory        pairs kept, 1..16; 2 * memory fields of ncomp x Nvox reals
 *                are allocated at the first call with that memory and kept
 *  max_iter      iteration cap (>= 1)
 *  rep_host      may be NULL; nr_iters = iterations, cg_iters = line-search
 *                trials, rejected = step halvings, restarts = skipped pairs,
 *                boundary_hits = pair resets, hv_products = 0, R = last alpha
 * The history is committed on convergence as in rve_solve_step.
 * RVE_ERR_ARG on a bad memory / max_iter; RVE_ERR_NOT_CONVERGED (state kept,
 * history not committed) when max_iter is reached or the line search fails. */
rve_status rve_solve_step_lbfgs(rve_t, const double dE_host[6], const uint8_t free_mask_host[6],
                                int memory, int max_iter, rve_step_report* rep_host);

/* Effective (homogenised) secant stiffness of the cell at the current damage
 * field D (the state's, or the one set by rve_set_damage), for the
 * stiffness-loss measure ||C_bar|| / ||C_bar_0|| of the ASR example
 * (Sec. 3.3).  For every Mandel unit mean strain e_j, with every mean
 * component strain-controlled, the fluctuation x_j solving
 * G : (1-D) C : (e_j + x_j) = 0 is found by Steihaug CG without a radius
 * (Algorithm 1 on the product of Eq. (8)) to |r| <= tol |G:(1-D)C:e_j|;
 * C_bar column j = <(1-D) C : (e_j + x_j)>.
 *  tol             relative CG tolerance, in (0, 1)
 *  max_cg          CG iteration cap per column (>= 1)
 *  Cbar_host       ncomp x ncomp doubles, row-major, Mandel (written)
 *  cg_iters_host   total CG iterations (may be NULL)
 * The state, the free mask, the trust radius and the options are left as
 * they were; the Hessian-vector counter counts the products.  Synchronises
 * the stream.  RVE_ERR_ARG on bad arguments; RVE_ERR_NOT_CONVERGED when a
 * column's CG reaches max_cg (or meets zero curvature on a fully damaged
 * cell). */
rve_status rve_effective_stiffness(rve_t, double tol, int max_cg, double* Cbar_host, int* cg_iters_host);

/* Per-pass device timing, for benchmarks (not part of the method).
 * Pass ids: 0 x-forward FFT with the fused tangent, 1 y-forward FFT,
 * 2 z-FFT + projection + inverse z-FFT, 3 y-inverse FFT, 4 x-inverse FFT,
 * 5 2D y-FFT + projection + inverse, 6 constitutive trial evaluation,
 * 7 CG vector updates.  rve_pass_timing(h, 1) starts (and resets) the
 * recording of CUDA events on the context's stream around every launch of
 * those kernels (up to 8192 launches; later ones are not timed; while it is
 * on, the host steps the Steihaug-CG iterations one at a time, since events
 * cannot be recorded inside the device-side loop -- same kernels, same
 * results);
 * rve_pass_timing(h, 0) stops it.  rve_pass_stats synchronises on the last
 * event and writes, for pass ids 0..n-1, the number of timed launches and
 * their summed device time in milliseconds. */
#define RVE_NPASS 8
rve_status rve_pass_timing(rve_t, int enable);
rve_status rve_pass_stats(rve_t, long long* counts_host, double* ms_host, int n);

/* Projection out = G : v (as rve_project, FP32 fields) for callers that must
 * not allocate device memory: code past a fixed-budget initialisation phase
 * (real-time or embedded loops, frameworks whose caching allocator owns all
 * device memory) and code that must not trigger the implicit device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  The paper has no
 * counterpart: this is a deployment variant of the projection.
 *  dims, ndim     grid as for rve_create; limit: ncomp*Ny*Nz*(Nx/2+1) <=
 *                 2087936 complex values (e.g. 80^3 in 3D, 1024^2 in 2D).
 *  v_dev, out_dev ncomp x Nvox FP32 device fields (may alias), caller-owned.
 *  free_mask_host stress-controlled mean components (NULL = none).
 *  stream         cudaStream_t (as void*); NULL = legacy default stream.
 * No context is needed and nothing is allocated: the scratch (axis tables
 * and half spectrum) lives in a fixed 16 MiB __device__ array that every GPU
 * loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.
 * Every call on a device shares the array and overwrites it (nothing in it
 * needs to start at zero); calls whose work overlaps on the GPU (different
 * streams, or host threads without ordering) race on it and must be
 * serialised by the caller.  Returns RVE_ERR_ARG (NULL pointer, bad dims,
 * grid over the limit) or RVE_ERR_CUDA; no message is stored.  A CUDA error
 * already pending on the calling thread when the call starts (from earlier
 * work) makes it return RVE_ERR_CUDA at once, launching nothing and leaving
 * that error pending for its owner (cudaGetLastError). */
rve_status rve_project_noalloc(const int dims[3], int ndim, const float* v_dev, float* out_dev,
                               const uint8_t free_mask_host[6], void* stream);

/* ------------------------------------------------------------------------
 * Batched solver: n RVEs of uneven sizes (2D and 3D may be mixed) advanced
 * in lockstep, FP32 fields.  Each step of the path (tangent + FFT passes +
 * projection, CG reductions and updates, constitutive update, scalar
 * control) is one persistent launch over all members, pulling (member,
 * block) work items from a counter; the inner CG iteration is replayed from
 * a captured CUDA graph.  Same method and results as n independent contexts.
 * ------------------------------------------------------------------------ */
typedef struct rve_batch_ctx* rve_batch_t;

/* dims: n*3 ints (Nx, Ny, Nz per member; Nz ignored in 2D); ndims: n ints;
 * phase_ids_dev: host array of n device pointers (Nvox_i uint8 each, copied);
 * phases shared by all members; opts as for rve_create (precision 32 only).
 * 1 <= n <= 256. */
rve_status rve_batch_create(int n, const int* dims_host, const int* ndims_host,
                            const uint8_t* const* phase_ids_dev, const rve_phase* phases_host,
                            int nphase, const rve_solver_opts* opts_host, void* stream,
                            rve_batch_t* out);
/* One load step of Algorithm 2 for every member: dE_host n*6 (Mandel, per
 * member), free_mask_host n*6 or NULL (keep), reps_host n reports.
 * Returns RVE_ERR_NOT_CONVERGED if any member hit max_nr (its history is
 * not committed; converged members commit theirs). */
rve_status rve_batch_solve_step(rve_batch_t, const double* dE_host, const uint8_t* free_mask_host,
                                rve_step_report* reps_host);
/* One batched Hessian-vector product out_i = G:((1-D_i)C:v_i) on every
 * member (host arrays of n device pointers, ncomp*Nvox_i floats each). */
rve_status rve_batch_hessp(rve_batch_t, const float* const* v_dev, float* const* out_dev);
/* Frozen damage of member i (Nvox_i floats), as rve_set_damage. */
rve_status rve_batch_set_damage(rve_batch_t, int i, const float* damage_dev);
/* State of member i, as rve_get_state (any pointer may be NULL). */
rve_status rve_batch_get_state(rve_batch_t, int i, float* strain_dev, float* kappa_dev,
                               float* stress_dev, float* damage_dev);
/* Back to the unloaded state (eps = 0, kappa_n = 0) for every member; the
 * trust radii are kept. */
rve_status rve_batch_reset(rve_batch_t);
/* Schedule autotuner of the batched spectral passes (not part of the
 * method): times one batched Hessian-vector product of every member for a
 * few schedules -- each member's x / y / z tile divided by 1, 2 or 4, and
 * every axis's radix order natural or reversed -- `reps` times each (1..1000),
 * by coordinate search (a candidate must be 2 % faster), and keeps the
 * fastest for all later calls.  base_ms_host / best_ms_host (may be NULL):
 * time per product of the default schedule and of the chosen one;
 * schedule_host (may be NULL, 4 ints): x, y, z divisors and 1 if the radix
 * order is reversed.  Overwrites the CG scratch vectors, so call it between
 * load steps; synchronises the stream. */
rve_status rve_batch_autotune(rve_batch_t, int reps, double* base_ms_host, double* best_ms_host,
                              int* schedule_host);
/* Install one schedule by hand (4 ints as above; divisors 1, 2 or 4). */
rve_status rve_batch_set_schedule(rve_batch_t, const int* schedule_host);
const char* rve_batch_last_error(rve_batch_t);
long long rve_batch_hv_count(rve_batch_t);
long long rve_batch_launch_count(rve_batch_t);
void rve_batch_destroy(rve_batch_t);

/* ------------------------------------------------------------------------
 * Learned warm start: a spectral neural operator that proposes the next
 * load step's strain-fluctuation increment (the paper has no learned part;
 * the proposal only seeds the trust-region solve, which still decides
 * convergence).  Inputs channels last [B][Nz][Ny][Nx][cin] (phase one-hot,
 * damage, previous two fluctuation increments), output [..][cout].
 * Network: lift, `layers` Fourier layers of width 32 (retained modes kx in
 * [0, modes), ky, kz in [-modes/2, modes/2); per-mode real 64 x 64 maps of
 * the (Re, Im) channel pairs, BF16; GELU between layers), projection.  All
 * contractions on the tensor cores (BF16 operands, FP32 accumulation).
 * Parameters are one packed FP32 vector: Wl (cin x 32, [in][out]), bl (32),
 * per layer W (32 x 32, [in][out]), b (32), R (modes^3 x 64 x 64), then Wq
 * (32 x cout, [in][out]), bq (cout).
 * ------------------------------------------------------------------------ */
typedef struct rve_fno_ctx* rve_fno_t;
rve_status rve_fno_create(int cin, int width, int cout, int layers, int modes, unsigned long long seed,
                          void* stream, rve_fno_t* out);
long long rve_fno_param_count(rve_fno_t);
/* Replace the parameters (host, packed) and reset the optimiser state. */
rve_status rve_fno_set_params(rve_fno_t, const float* params_host);
/* Copy out the parameters and / or the last gradient (host, packed; NULL skips). */
rve_status rve_fno_get_params(rve_fno_t, float* params_host, float* grad_host);
/* y = net(x) for batch <= 8 samples of grid dims (Nx, Ny, Nz); Nx >= 2 modes
 * (no retained mode at or above the real axis' Nyquist index), Ny, Nz >= modes. */
rve_status rve_fno_forward(rve_fno_t, int batch, const int dims[3], const float* x_dev, float* y_dev);
/* Mean-squared-error loss against targets t and its gradient (kept for the
 * next rve_fno_adam_step, readable with rve_fno_get_params).  Synchronises. */
rve_status rve_fno_loss_grad(rve_fno_t, int batch, const int dims[3], const float* x_dev, const float* t_dev,
                             double* loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. */
rve_status rve_fno_adam_step(rve_fno_t, double lr);
/* Build the input features of one sample from solver fields (FP32 SoA):
 * phase ids, damage (may be NULL), previous two fluctuation increments
 * (6 x Nvox each, may be NULL) scaled by `scale`, and, in channel 15 when
 * cin >= 16, the history variable kappa (may be NULL) times kappa_scale.
 * Needs cin >= 15. */
rve_status rve_fno_pack_features(rve_fno_t, const int dims[3], const uint8_t* phase_dev, const float* damage_dev,
                                 const float* kappa_dev, float kappa_scale, const float* d1_dev, const float* d2_dev,
                                 float scale, float* x_dev);
/* Channels-last output of one sample -> SoA Mandel field:
 * out = base + scale * y (base, a SoA field, may be NULL; with base = the
 * last fluctuation increment the network predicts the change of the
 * increment). */
rve_status rve_fno_unpack_output(rve_fno_t, const int dims[3], const float* y_dev, float scale, const float* base_dev,
                                 float* out_dev);
/* SoA Mandel fields (cout x Nvox) -> channels-last training target
 * t = scale * (field - base) [Nz][Ny][Nx][cout] (base may be NULL; the
 * inverse of rve_fno_unpack_output). */
rve_status rve_fno_pack_target(rve_fno_t, const int dims[3], const float* field_dev, const float* base_dev, float scale,
                               float* t_dev);
/* Fluctuation increment between two converged FP32 strain fields (cout x
 * Nvox each): out = eps_new - eps_old - dE (dE uniform per Mandel component,
 * the applied mean-strain increment of the step). */
rve_status rve_fno_increment(rve_fno_t, const int dims[3], const float* eps_new_dev, const float* eps_old_dev,
                             const double dE_host[6], float* out_dev);
const char* rve_fno_last_error(rve_fno_t);
long long rve_fno_launch_count(rve_fno_t);
void rve_fno_destroy(rve_fno_t);

/* Message of the last error on this context (static storage; never NULL). */
const char* rve_last_error(rve_t);

/* Number of Hessian-vector products and of kernel launches issued by this
 * context since creation (counters for benchmarks). */
long long rve_hv_count(rve_t);
long long rve_launch_count(rve_t);
/* Number of times this context waited on its stream to read the device
 * scalars that steer Algorithms 1 and 2 (a counter for benchmarks).  The
 * Steihaug-CG iterations run on the device as a CUDA graph whose WHILE node
 * repeats the iteration until an exit or a restart, so a solve waits about
 * twice plus once per restart, not once per iteration; with per-pass timing
 * on (rve_pass_timing) the host steps the iterations and waits after each. */
long long rve_sync_count(rve_t);

/* Where the Steihaug-CG iterations are driven from, for benchmarks and
 * tests (not part of the method): 1 (default) on the device, as the graph
 * loop described at rve_sync_count; 0 from the host, one launch sequence
 * and one wait per iteration.  Both run the same kernels in the same order
 * and give identical results. */
rve_status rve_set_device_loop(rve_t, int enable);

/* Free the context and its workspaces.  NULL is ignored. */
void rve_destroy(rve_t);

#ifdef __cplusplus
}
#endif

#endif /* RVE_H */
