/*
 * tomo.h -- C ABI of the exact-gradient path of SIMP compliance minimisation on a
 * structured hex8 voxel grid, built for NVIDIA GB300 (sm_103a).
 *
 * The problem (Eq. 4, Section III-D of "Speeding up Computational Morphogenesis with Online
 * Neural Synthetic Gradients"): minimise the compliance c = f^T u(z) subject to
 * v^T P z <= V_max and 0 <= z_i <= 1, where u(z) solves K(P z) u = f (the state equation
 * r = K u - f = 0), P is the density filter and K(rho) = sum_e h E_e(rho_e) K0 with the
 * modified SIMP modulus E_e = Emin + rho_e^p (E0 - Emin).  Its gradient is Eq. 5,
 * g_i = -u^T (dK/dz_i) u, and the volume gradient is P^T v (Section III-D).  The design is
 * updated by the optimality-criteria (OC) method (Section III-D, Algorithm 1).
 *
 * Layout (all arrays, host or device):
 *   elements  e = i + nx*(j + ny*k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz  (x fastest)
 *   nodes     n = i + (nx+1)*(j + (ny+1)*k)
 *   nodal vectors are structure-of-arrays: component c (0=x, 1=y, 2=z) of node n at
 *   index c*N_n + n, N_n = (nx+1)(ny+1)(nz+1).
 *
 * Ownership: the caller owns every array passed in or out; the library copies the
 * descriptor's host arrays at creation and owns its internal state (multigrid hierarchy,
 * scratch vectors, constants) until tomo_destroy_grid.
 *
 * Pointers: every array argument may be a device pointer (cudaMalloc / torch tensor on
 * the grid's device) or a host pointer (pageable or pinned).  Host arrays are staged
 * through internal device buffers; the call then synchronises the grid's stream before it
 * returns.  With device pointers all work is queued on the grid's stream and the call
 * returns without waiting, except where a host scalar is written (compliance, change,
 * solve info), which waits for the stream.
 *
 * Precision: a grid is created in one precision.  TOMO_FP64 grids take the *_d entry
 * points (double arrays) and compute everything in FP64.  TOMO_FP32 grids take the float
 * entry points: matrix-free products and multigrid smoothing in FP32, the CG iterate kept
 * as an unevaluated float pair (about 48 significant bits), inner products as per-thread
 * float pairs (TwoSum) summed in FP64 across threads, residual replacement, the compliance
 * and the OC volume sums in FP64.  Calling an entry point of the other precision returns
 * TOMO_EINVAL.
 *
 * Errors: every call returns a tomo_status.  Nothing aborts or traps; after an error the
 * handle stays valid and tomo_last_error() describes the most recent failure on it.
 * Calls on one handle are not thread-safe; distinct handles are independent.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tomo_grid tomo_grid; /* opaque, owned by the library */
typedef struct tomo_batch tomo_batch; /* opaque: a set of grids evaluated together */

typedef enum {
  TOMO_OK = 0,
  TOMO_EINVAL = 1,   /* bad argument, size, layout or precision */
  TOMO_ENOMEM = 2,   /* device or host allocation failed */
  TOMO_ENOCONV = 3,  /* CG stopped at maxit or broke down (p^T A p <= 0) */
  TOMO_ENAN = 4,     /* a NaN/Inf appeared in the iteration */
  TOMO_ETIMEOUT = 5, /* a bounded device wait ran out */
  TOMO_ECUDA = 6,    /* a CUDA runtime call failed (message in tomo_last_error) */
  TOMO_EBUSY = 7     /* the handle is in use by an unfinished call */
} tomo_status;

enum { TOMO_FP64 = 0, TOMO_FP32 = 1 };
enum { TOMO_PRECOND_MG = 0, TOMO_PRECOND_JACOBI = 1 };

typedef struct {
  int32_t iters;       /* CG iterations taken */
  double rel_res;      /* ||r||_2 / ||f||_2 of the recursively updated residual at exit */
  int32_t status;      /* tomo_status of the solve */
  int32_t mg_levels;   /* multigrid levels used (1 for Jacobi) */
} tomo_solve_info;

typedef struct {
  int32_t nx, ny, nz;   /* elements per axis, each >= 1 */
  double h;             /* element edge length (> 0); K_e = h E_e K0, v_e = h^3 */
  double E0, Emin;      /* solid and void moduli, E0 > Emin >= 0 */
  double nu;            /* Poisson ratio, -1 < nu < 0.5 */
  double penal;         /* SIMP exponent p >= 1 */
  double rmin;          /* filter radius in element units (cone weights rmin - dist) */
  const uint8_t* fixed_dof; /* host, 3*N_n, SoA; nonzero = displacement fixed to 0 */
  const double* f;      /* host, 3*N_n, SoA load vector */
  int32_t precision;    /* TOMO_FP64 | TOMO_FP32 */
  int32_t precond;      /* TOMO_PRECOND_MG (default) | TOMO_PRECOND_JACOBI */
  double rtol;          /* CG stop: ||r|| <= rtol ||f||; <= 0 selects 1e-6 */
  int32_t maxit;        /* CG iteration cap; <= 0 selects 2000 */
  int32_t mg_levels;    /* multigrid levels; <= 0 coarsens until the coarsest grid is small */
  int32_t smoother_degree; /* Chebyshev degree per pre/post smoothing, fine level; <= 0: 2 */
  int32_t coarse_degree;   /* the same on the coarser levels; <= 0: smoother_degree */
  double cheb_ratio;    /* smoothing interval [lmax/ratio, lmax] of D^-1 K; <= 1 selects 20 */
  double cheb_lmax;     /* lmax; <= 0 selects the element bound max eig(diag(K0)^-1 K0), which
                           bounds eig(D^-1 K) on any grid (5.32 for nu = 0.3) */
  int32_t rr_every;     /* residual replacement r = f - K x (evaluated in FP64) every rr_every
                           iterations; 0 selects 50, < 0 off */
  void* stream;         /* cudaStream_t for all work on this grid; NULL = legacy default */
} tomo_grid_desc;

/* Fill *desc with defaults (no arrays, FP32, MG, rtol 1e-6, maxit 2000, auto levels,
 * degree 2, residual replacement every 50 iterations, E0=1, Emin=1e-9, nu=0.3, p=3,
 * rmin=1.5, h=1). */
void tomo_default_desc(tomo_grid_desc* desc);

/* Validate the descriptor, copy its host arrays, build K0 (Section III-D, hex8, E = 1,
 * unit cube), the filter weights, the multigrid hierarchy and all scratch on the current
 * CUDA device.  *out receives the handle.  TOMO_EINVAL on bad sizes or parameters,
 * TOMO_ENOMEM if device memory runs out. */
tomo_status tomo_create_grid(const tomo_grid_desc* desc, tomo_grid** out);

/* Synchronise the grid's stream and release everything the handle owns. NULL is a no-op. */
tomo_status tomo_destroy_grid(tomo_grid* grid);

/* Rebind the grid to another stream (cudaStream_t); later calls queue there. */
tomo_status tomo_set_stream(tomo_grid* grid, void* stream);

/* Density filter of Eq. 4 (Section III-D): transpose = 0 computes out = P in = (H in)/Hs,
 * transpose != 0 computes out = P^T in = H (in/Hs).  H_ij = max(0, rmin - |x_i - x_j|)
 * over element centroids, Hs = H 1 truncated at the domain boundary.  in/out: N_el
 * element arrays; they must not overlap. */
tomo_status tomo_filter(tomo_grid* grid, const float* in, float* out, int transpose);
tomo_status tomo_filter_d(tomo_grid* grid, const double* in, double* out, int transpose);

/* Two-scale coarse-graining (Section III-C; Algorithm 1, first step of every iteration):
 * z_coarse[I + cx (J + cy K)] = mean of z over the block of elements
 * [I*block, (I+1)*block) x [J*block, ...) x [K*block, ...), with cx = ceil(nx / block),
 * cy = ceil(ny / block), cz = ceil(nz / block); a block cut by the domain boundary averages
 * the elements it holds.  The coarse state of Algorithm 1 (K_C(z_C) u_C = f_C) is a
 * tomo_solve on a grid created for the coarse mesh (element edge block*h) with rho = z_C.
 * z: N_el elements of this grid; z_coarse: cx*cy*cz elements (caller-owned, host or
 * device, must not overlap z).  block < 1 returns TOMO_EINVAL.  Sums are accumulated in
 * double. */
tomo_status tomo_coarse_grain(tomo_grid* grid, const float* z, int32_t block, float* z_coarse);
tomo_status tomo_coarse_grain_d(tomo_grid* grid, const double* z, int32_t block,
                                double* z_coarse);

/* y = K(rho) x on the free DOFs (fixed rows and the fixed entries of x are zero), with
 * K(rho) = sum_e h E_e K0 and E_e = Emin + rho_e^p (E0 - Emin) (state equation of Eq. 4).
 * rho: N_el physical densities in [0,1]; x, y: 3*N_n nodal vectors (SoA), no overlap. */
tomo_status tomo_apply_stiffness(tomo_grid* grid, const float* rho, const float* x, float* y);
tomo_status tomo_apply_stiffness_d(tomo_grid* grid, const double* rho, const double* x, double* y);

/* Residual of the state equation of Eq. 4: r = f - K(rho) u on the free DOFs (0 on fixed
 * DOFs).  FP32 grids take u as the unevaluated pair u + u_lo (u_lo may be NULL), the form
 * in which the solver keeps its iterate.  rho: N_el; u, u_lo, r: 3*N_n. */
tomo_status tomo_residual(tomo_grid* grid, const float* rho, const float* u, const float* u_lo,
                          float* r);
tomo_status tomo_residual_d(tomo_grid* grid, const double* rho, const double* u, double* r);

/* Solve K(rho) u = f (state equation of Eq. 4, Section III-D) by CG preconditioned with a
 * geometric-multigrid V-cycle (or Jacobi), to ||r|| <= rtol ||f||.  rho: N_el physical
 * densities.  u: 3*N_n; on entry a warm start (fixed entries ignored), on exit the
 * solution.  info (may be NULL) receives iterations, residual and status.  Returns
 * TOMO_ENOCONV if maxit was reached, TOMO_ENAN on a NaN.  u holds the last iterate in
 * both cases. */
tomo_status tomo_solve(tomo_grid* grid, const float* rho, float* u, tomo_solve_info* info);
tomo_status tomo_solve_d(tomo_grid* grid, const double* rho, double* u, tomo_solve_info* info);

/* Compliance and its sensitivity (Eq. 4 objective, Eq. 5 with the SIMP chain rule):
 * *compliance = f^T u (host or device double), and
 * dc[e] = -p rho_e^(p-1) (E0 - Emin) h u_e^T K0 u_e  (derivative w.r.t. rho_e).
 * rho: N_el, u: 3*N_n, dc: N_el.  compliance or dc may be NULL to skip them. */
tomo_status tomo_sensitivity(tomo_grid* grid, const float* rho, const float* u,
                             double* compliance, float* dc);
tomo_status tomo_sensitivity_d(tomo_grid* grid, const double* rho, const double* u,
                               double* compliance, double* dc);

/* One optimality-criteria update (Section III-D): with B_e = max(-dcdz_e, 0)/(lam dvdz_e),
 * z_new = clamp(z sqrt(B_e), max(0, z - move), min(1, z + move)), lam chosen so that
 * sum_e dvdz_e z_new_e = volfrac * N_el * h^3 (the filtered volume v^T P z_new of Eq. 4),
 * located to a relative bracket width of 1e-10 (at most 2^100).  *change (host or device
 * double, may be NULL) = max_e |z_new_e - z_e|.  All arrays N_el; z_new must not overlap
 * the inputs. */
tomo_status tomo_oc_step(tomo_grid* grid, const float* z, const float* dcdz, const float* dvdz,
                         double volfrac, double move, float* z_new, double* change);
tomo_status tomo_oc_step_d(tomo_grid* grid, const double* z, const double* dcdz,
                           const double* dvdz, double volfrac, double move, double* z_new,
                           double* change);

/* tomo_oc_step without any allocation, for callers that may not allocate device memory
 * (runtimes that own all device memory through their own pool and forbid driver
 * allocations, loops that cannot afford an allocation's implicit synchronisation).  The
 * paper has no counterpart: this is a deployment variant of tomo_oc_step for FP32 data,
 * computing the same update with the same multiplier search.
 *   n_el:   number of design variables, 1 <= n_el <= 4,194,304 (larger: TOMO_EINVAL);
 *   h:      element edge (V_max = volfrac * n_el * h^3);
 *   z, dcdz, dvdz, z_new: float arrays of n_el entries in device memory of the CURRENT
 *           device (host pointers or another GPU's memory: TOMO_EINVAL);
 *   change: double in device memory of the current device receiving max |z_new - z|, or
 *           NULL;
 *   stream: cudaStream_t of the current device the work is queued on (NULL = legacy
 *           default; a stream of another device: TOMO_EINVAL); nothing waits.
 * Scratch: a static device array of about 0.5 MiB inside this library, held by every GPU
 * that loads it until the process exits.  The first call on a device resolves that array's
 * device address (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  All calls share the array: calls that overlap on the GPU
 * (different streams, or several devices' worth of work on one) race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or other allocating call is made.
 * Errors: TOMO_EINVAL / TOMO_ECUDA, described by tomo_last_error(NULL). */
tomo_status tomo_oc_step_noalloc(int64_t n_el, double h, const float* z, const float* dcdz,
                                 const float* dvdz, double volfrac, double move, float* z_new,
                                 double* change, void* stream);

/* One exact-gradient evaluation (Algorithm 1, exact branch; Eq. 4-5): rho = P z,
 * E = Emin + rho^p (E0 - Emin), solve K u = f from a zero start, *compliance = f^T u,
 * dcdz = P^T dc/drho, dvdz = P^T v.  z, dcdz, dvdz: N_el.  dvdz may be NULL (then it is not
 * computed).  The solution u stays inside the handle (tomo_get_displacement). */
tomo_status tomo_gradient(tomo_grid* grid, const float* z, double* compliance, float* dcdz,
                          float* dvdz, tomo_solve_info* info);
tomo_status tomo_gradient_d(tomo_grid* grid, const double* z, double* compliance,
                            double* dcdz, double* dvdz, tomo_solve_info* info);

/* General objective through the adjoint (Eq. 3), for a linear functional of the state,
 * J = l^T u (e.g. a displacement or a weighted set of them; dJ/dz = 0 explicitly): solves
 * K u = f and K lambda = l (dr/du = K is symmetric), then *J = l^T u and
 * djdz = P^T dJ/drho with dJ/drho_e = -p rho_e^(p-1) (E0 - Emin) h lambda_e^T K0 u_e.
 * Compliance is the case l = f (lambda = u).  z, djdz: N_el; l: 3*N_n SoA, its fixed
 * entries are ignored.  info_u / info_l (may be NULL) report the two solves; both start
 * from zero.  The state u stays in the handle (tomo_get_displacement). */
tomo_status tomo_adjoint_gradient(tomo_grid* grid, const float* z, const float* l, double* J,
                                  float* djdz, tomo_solve_info* info_u,
                                  tomo_solve_info* info_l);
tomo_status tomo_adjoint_gradient_d(tomo_grid* grid, const double* z, const double* l,
                                    double* J, double* djdz, tomo_solve_info* info_u,
                                    tomo_solve_info* info_l);

/* on != 0: later tomo_gradient calls on this grid start CG from the displacement of the
 * previous solve on the grid (when there is one) instead of zero; the starting residual
 * f - K u is evaluated in FP64.  Useful along an optimisation run, where u changes little
 * between iterations; the result is the same solve to the same tolerance.  on = 0 (the
 * default) restores the zero start. */
tomo_status tomo_set_warm_start(tomo_grid* grid, int32_t on);

/* Smoother of the multigrid preconditioner (Section III-D names multigrid as the
 * alternative to Jacobi-PCG; the smoother is this library's choice): Chebyshev-Jacobi of
 * degree fine_degree on the finest level and coarse_degree on the coarser ones (1..16), on
 * [lam / ratio, lam] of D^-1 K with lam the element bound (ratio > 1).  Any setting gives
 * the same solve to the same tolerance; the number of CG iterations and the time per
 * iteration change.  tomo_set_smoother waits for the grid's stream and sets the captured
 * CG loop aside (kept for up to 8 settings and reused when the setting returns; a new one
 * is captured at the next solve); EINVAL for degrees or ratio out of range.
 * tomo_get_smoother: any pointer may be NULL. */
tomo_status tomo_set_smoother(tomo_grid* grid, int32_t fine_degree, int32_t coarse_degree,
                              double ratio);
tomo_status tomo_get_smoother(const tomo_grid* grid, int32_t* fine_degree,
                              int32_t* coarse_degree, double* ratio);

/* Upper end lam of the smoothing interval [lam / ratio, lam] of D^-1 K (Section III-D's
 * multigrid; the interval is this library's choice).  lam <= 0 selects the element bound
 * max eig(diag(K0)^-1 K0), which bounds the spectrum of any design (the default); a smaller
 * lam (at least a quarter of the bound, else EINVAL) smooths the actual spectrum, which on
 * designs without isolated elements ends near 3.1-3.9, better and saves CG iterations.  If a
 * solve with lam below the bound fails (the interval misses the top of the spectrum: the
 * preconditioner is not positive or CG does not converge), the solve is redone from zero at
 * the element bound and the grid keeps the bound; tomo_get_smoother_bound counts these
 * fallbacks.  Like tomo_set_smoother it waits for the grid's stream and sets the captured CG
 * loop aside.  tomo_get_smoother_bound: any pointer may be NULL. */
tomo_status tomo_set_smoother_bound(tomo_grid* grid, double lam);
/* Cycle shape of the multigrid preconditioner: bit l of w_levels set makes the cycle
 * correct twice from level l + 1 at level l (x += P M P^T (b - A x) once more after the
 * first correction, before the post-smoothing): a W-cycle at that level, which can save CG
 * iterations where the rediscretised coarse operators are weak (designs evolved towards
 * 0/1 densities) at the price of running the coarser levels twice.  0 (the default) is the V-cycle.  Bits of the two coarsest levels have no
 * effect (the level above the coarsest corrects exactly).  The cycle stays symmetric, so it
 * remains a valid CG preconditioner.  A grid with W-cycle levels runs alone in a batch (one
 * grid per worker stream, not lockstep).  Like tomo_set_smoother it waits for the grid's
 * stream and sets the captured loop aside.  tomo_get_cycle reads the mask. */
tomo_status tomo_set_cycle(tomo_grid* grid, uint32_t w_levels);
tomo_status tomo_get_cycle(const tomo_grid* grid, uint32_t* w_levels);
/* Coarse tail (FP32 multigrid grids): with on != 0 the V-cycle runs its levels from the
 * first one below the finest with at most 4096 elements down to the coarsest and back
 * (smoothing, residual, transfers, coarsest solve) as ONE launch of a thread-block cluster,
 * its passes separated by cluster barriers, instead of about six launches per level.  The
 * operator is the same (the launched levels' definitions); only the order in which a
 * node's element contributions are added differs, so results agree to rounding.  Levels
 * with W-cycle bits at or below the entry level keep the launched form.  No effect on grids
 * without such a level (tomo_get_coarse_tail reports 0) or on lockstep batches.  Like
 * tomo_set_smoother it waits for the grid's stream and drops the captured loops.
 * tomo_get_coarse_tail: the entry level in use, 0 when off. */
tomo_status tomo_set_coarse_tail(tomo_grid* grid, int32_t on);
tomo_status tomo_get_coarse_tail(const tomo_grid* grid, int32_t* level);
tomo_status tomo_get_smoother_bound(const tomo_grid* grid, double* lam, double* element_bound,
                                    int64_t* fallbacks);

/* Smoother autotuner.  On the design z (N_el, host or device; filtered and turned into the
 * material as tomo_gradient does) it times the state solve from a zero start for each
 * candidate (pairs[2k], pairs[2k+1]) = (fine_degree, coarse_degree), k < n (1..64), at the
 * grid's current ratio, bound and cycle: one untimed solve (skipped when the grid kept that
 * candidate's captured loop from an earlier use: a grid keeps the loops of up to 8 smoother
 * settings), then reps (1..16) solves timed with CUDA events on the grid's stream, the
 * median kept.  pairs == NULL: the built-in stages, 23 candidates (n ignored; results needs
 * room for 23): the degree pairs (2,2) (2,3) (2,4) (1,3) (1,4) (1,6), each at 1, 0.75 and
 * 0.68 times the element bound, as V-cycles (18); the fastest of these with a W-cycle at
 * level 1 and at levels 1 and 2 (tomo_set_cycle masks 2 and 6); the fastest so far with the
 * smoothing interval [lam/ratio, lam] at ratios 12, 30 and 50.  Candidates are timed
 * without the bound fallback of the solves (a candidate that fails is only marked failed).
 * The fastest candidate that converges becomes the grid's smoother and cycle; results[k]
 * (may be NULL) holds each candidate's median milliseconds (-1 when it failed or its stage
 * did not run), iterations, status, bound, cycle mask and ratio; *best (may be NULL) its
 * index.  If no candidate converges the grid keeps its previous setting and ENOCONV is
 * returned.  The grid's displacement is left as the last trial's.
 * tomo_autotune_smoother_multi: the same on nz (1..16) designs z[0..nz): a candidate's time
 * is the sum of its medians over the designs, its iterations the largest count, and it
 * fails if it fails on any design (a setting for a family of designs rather than one). */
typedef struct {
  int32_t fine_degree, coarse_degree;
  int32_t iters;
  int32_t status;
  double ms;
  double lam;         /* upper end of the smoothing interval the candidate used */
  uint32_t w_levels;  /* the candidate's cycle (tomo_set_cycle mask) */
  uint32_t reserved;
  double ratio;       /* the candidate's interval ratio (lam / lower end) */
} tomo_tune_result;
tomo_status tomo_autotune_smoother(tomo_grid* grid, const float* z, const int32_t* pairs,
                                   int32_t n, int32_t reps, tomo_tune_result* results,
                                   int32_t* best);
tomo_status tomo_autotune_smoother_d(tomo_grid* grid, const double* z, const int32_t* pairs,
                                     int32_t n, int32_t reps, tomo_tune_result* results,
                                     int32_t* best);
tomo_status tomo_autotune_smoother_multi(tomo_grid* grid, const float* const* z, int32_t nz,
                                         const int32_t* pairs, int32_t n, int32_t reps,
                                         tomo_tune_result* results, int32_t* best);
tomo_status tomo_autotune_smoother_multi_d(tomo_grid* grid, const double* const* z,
                                           int32_t nz, const int32_t* pairs, int32_t n,
                                           int32_t reps, tomo_tune_result* results,
                                           int32_t* best);

/* Copy the displacement of the last tomo_gradient / tomo_solve on this grid to u
 * (3*N_n, host or device). */
tomo_status tomo_get_displacement(tomo_grid* grid, float* u);
tomo_status tomo_get_displacement_d(tomo_grid* grid, double* u);

/* Grid counts: n_el, n_nodes, number of multigrid levels; any pointer may be NULL. */
tomo_status tomo_get_counts(const tomo_grid* grid, int64_t* n_el, int64_t* n_nodes,
                            int32_t* mg_levels);

/* Number of kernels this grid has launched since creation (kernels of the device-side CG
 * loop counted once per executed iteration). */
tomo_status tomo_get_launch_count(const tomo_grid* grid, int64_t* launches);

/* Timing for roofline and phase reports.  enable bit 0: the library brackets every launch
 * of the fine-level matrix-free kernels (products and smoother steps) with CUDA events on
 * the grid's stream and accumulates their count, total milliseconds and algorithmic DRAM
 * bytes (inputs read once plus outputs written once); the CG loop is then issued from the
 * host (same kernels, same order) because event records cannot sit inside the device-side
 * loop; the host issues iterations four at a time, so the launches enqueued after the
 * solve stopped (the rest of the last iteration after its convergence test, and up to
 * three further iterations) return at once on the device flag: they are left out of the
 * totals and the level tables.  tomo_profile_read waits for the stream, returns the totals
 * since the last reset and resets them.  enable bit 1: events at phase boundaries only (device-side loop kept);
 * tomo_profile_phases returns the accumulated milliseconds of ms[0] filter + material,
 * ms[1] multigrid level setup, ms[2] CG solve, ms[3] compliance + sensitivity, ms[4] filter
 * adjoints, ms[6] OC step (ms[5] unused) and the number of gradient calls, then resets. */
tomo_status tomo_profile_enable(tomo_grid* grid, int enable);
tomo_status tomo_profile_phases(tomo_grid* grid, double* ms, int64_t* calls);
/* With enable bit 0 set, every kernel of the multigrid preconditioner is also timed and
 * binned by level: after tomo_profile_read, ms[l] / launches[l] (l < max_levels) hold the
 * device time and launch count of level l (level 0: the fine-level products only), then
 * reset. */
tomo_status tomo_profile_levels(tomo_grid* grid, double* ms, int64_t* launches, int max_levels);
tomo_status tomo_profile_read(tomo_grid* grid, int64_t* launches, double* total_ms,
                              double* algorithmic_bytes);

/* Batches of independent grids (uneven sizes allowed), evaluated together.  The paper
 * optimises one design at a time; a batch serves many small problems at once on one GPU.
 * tomo_batch_create: workers = number of concurrent host threads and CUDA streams (<= 0:
 * 8, at most 64), created on the device current at the call; every grid of the batch must
 * live on that device.  tomo_batch_append: adds a grid (not owned; it must outlive its use in
 * the batch and must not be used elsewhere while a batch call runs).  tomo_batch_gradient:
 * tomo_gradient on every grid i with z[i], &compliance[i], dcdz[i], dvdz[i] (dvdz or any
 * dvdz[i] may be NULL), info[i] (info may be NULL); FP32 grids only.
 * Lockstep mode (the default): filtering and level setup run per grid on the worker
 * streams, then one CG loop advances all grids together, every phase of an iteration (the
 * product, the vector updates, each multigrid level's smoothing, transfers and coarsest
 * solve) one launch for all grids, captured once as a device-side graph loop and reused
 * until the next tomo_batch_append; then the sensitivities run per grid.  It needs grids
 * with the multigrid preconditioner, the same smoother degrees, residual-replacement
 * interval and Poisson ratio, and profiling off; other batches, and batches with lockstep
 * off (tomo_batch_set_lockstep(batch, 0)), run each grid in order on one worker stream.
 * One grid per stream, each grid runs exactly the launches of its own tomo_gradient and
 * its result is bitwise the one it gives alone.  In lockstep the products' z-chunks are
 * chosen for the batch as a whole (one wave of CTAs for all grids), which changes only the
 * order in which the fused CG dots add their block partials: results agree with the grid
 * alone to rounding (same tolerance as any two runs to rtol) and are reproducible for the
 * same batch.  Returns when all grids are done; on failure the first failing grid's status, described by
 * tomo_batch_last_error.  tomo_batch_lockstep_runs: the number of tomo_batch_gradient calls
 * that ran in lockstep. */
tomo_status tomo_batch_create(int32_t workers, tomo_batch** out);
tomo_status tomo_batch_append(tomo_batch* batch, tomo_grid* grid);
tomo_status tomo_batch_size(const tomo_batch* batch, int32_t* count);
tomo_status tomo_batch_set_lockstep(tomo_batch* batch, int32_t on);
tomo_status tomo_batch_lockstep_runs(const tomo_batch* batch, int64_t* runs);
/* Phases of the last lockstep call, milliseconds: ms[0] host time to issue the per-grid
 * steps before the loop (filter, material, level setup, CG start), ms[1] device time from
 * their end to the end of the first V-cycle and search direction, ms[2] the CG loop,
 * ms[3] the read-back of the grids' CG scalars, ms[4] host time of the per-grid steps after
 * the loop (results, sensitivities, filter adjoints, up to the last stream's completion). */
tomo_status tomo_batch_phase_times(const tomo_batch* batch, double* ms);
/* Persistent lockstep iteration (off by default).  With on = 1 (2: with phase timing, see
 * tomo_batch_persistent_phase_ns; other values TOMO_EINVAL), each CG iteration of the
 * lockstep loop runs as ONE cooperative launch instead of one launch per phase: the
 * batched launches of an iteration are recorded (kind, CTA count, parameter table), and a
 * kernel with as many CTAs as the device holds co-resident runs them as phases, CTA b
 * taking the recorded CTAs b, b + grid, ... of each phase, a grid-wide barrier between
 * phases.  Every grid sees the same blocks and the same order of dot partials as in the
 * launched loop, so the results are bitwise those of lockstep without it.  Where the device
 * cannot run the kernel cooperatively (or the loop cannot be captured with it), the
 * launched iteration is used; tomo_batch_persistent_info then reports ctas = 0.
 * tomo_batch_set_wait_limit: nanoseconds a CTA waits at a barrier for the others (default
 * 2e9; >= 0, else TOMO_EINVAL).  A wait that runs out stops every grid of the loop: their
 * tomo_batch_gradient results are TOMO_ETIMEOUT (info[i].status too), nothing is written
 * to compliance/dcdz of those grids, the next call starts afresh (no warm start from the
 * stopped iterate).  Both settings take effect at the next call (the loop is recaptured).
 * tomo_batch_persistent_info: CTAs and phases of the captured persistent iteration (0 and 0
 * when the loop in use is the launched one) and the number of calls that ran it; any
 * pointer may be NULL. */
tomo_status tomo_batch_set_persistent(tomo_batch* batch, int32_t on);
tomo_status tomo_batch_set_wait_limit(tomo_batch* batch, int64_t limit_ns);
tomo_status tomo_batch_persistent_info(const tomo_batch* batch, int32_t* ctas, int32_t* phases,
                                       int64_t* runs);
/* Phase timing of the persistent iteration, enabled by tomo_batch_set_persistent(batch, 2)
 * (which adds one grid barrier per launch): device ns spent in each phase over all CG
 * iterations of the latest call, as CTA 0 sees it (from the previous barrier's exit to this
 * phase's), ns[p] with the phase's kind kinds[p] for p < min(count, cap); *count = the
 * number of phases (0 without timing or when the loop in use is the launched one);
 * *launches (may be NULL) = the persistent launches timed.  Kinds: 0 product, 1 product +
 * p^T q, 2 residual, 3 Chebyshev step, 4 Chebyshev step + b^T x, 5 FP64 residual
 * replacement, 6 Jacobi start, 7 restriction, 8 prolongation, 9 coarsest solve, 10 CG x/r
 * update, 11 CG p update.  A phase followed by a continuation of its launch (more than 64
 * grids) reports 0, its time counted with the continuation.  Synchronises the device. */
tomo_status tomo_batch_persistent_phase_ns(tomo_batch* batch, int64_t* ns, int32_t* kinds,
                                           int32_t cap, int32_t* count, int64_t* launches);
/* Tiles of the lockstep loop's batched products: tile_rows thread rows per CTA (8: tiles of
 * 30 x 14 nodes, as a grid alone; 4: 30 x 6 nodes, which fit small grids' y extent better at
 * more halo per node) and the waves of resident CTAs (1..16) that the z-chunk length aims
 * at; default 8 and 4.  Only the order of the fused dots' block partials depends on them
 * (results agree to rounding).  The persistent iteration takes 8-row tiles (with 4 the
 * launched iteration runs).  TOMO_EINVAL for other values; the next call recaptures the
 * loop.  tomo_batch_autotune_tiles: on the designs z[i] (dcdz[i] receives the gradients) it
 * runs tomo_batch_gradient for each of the 6 candidates (8, 4 rows x 2, 4, 8 waves): one
 * untimed call, then reps (1..16) calls timed by the device time of the batched phase (the
 * first V-cycle and the CG loop), the median kept; the fastest becomes the batch's setting.
 * results[k] (may be NULL, room for 6): rows, waves, status and median ms (-1 if the call
 * failed); *best (may be NULL) its index.  Needs a batch that runs in lockstep (else
 * TOMO_EINVAL); if no candidate runs, the previous setting is kept and TOMO_ENOCONV is
 * returned (TOMO_ECUDA, and the search stops, after a CUDA error). */
typedef struct {
  int32_t tile_rows, waves;
  int32_t status, reserved;
  double ms;
} tomo_batch_tune_result;
tomo_status tomo_batch_set_tiles(tomo_batch* batch, int32_t tile_rows, int32_t waves);
tomo_status tomo_batch_get_tiles(const tomo_batch* batch, int32_t* tile_rows, int32_t* waves);
tomo_status tomo_batch_autotune_tiles(tomo_batch* batch, const float* const* z,
                                      float* const* dcdz, int32_t reps,
                                      tomo_batch_tune_result* results, int32_t* best);
tomo_status tomo_batch_gradient(tomo_batch* batch, const float* const* z, double* compliance,
                                float* const* dcdz, float* const* dvdz, tomo_solve_info* info);
tomo_status tomo_batch_destroy(tomo_batch* batch);
const char* tomo_batch_last_error(const tomo_batch* batch);

/* Request loop (serving): gradient and optimisation requests on design domains of
 * different sizes, run
 * by `workers` threads with one CUDA stream each, with grids kept resident on the device
 * per session and admission by device memory.  The paper has no counterpart (it optimises
 * one design at a time); the arithmetic of each request is tomo_gradient's.
 * tomo_server_create: budget_bytes = device memory the resident grids may hold (their
 *   estimated footprint, tomo_estimate_device_bytes).
 * tomo_server_submit: desc (FP32; fixed_dof, f and z are copied), session >= 0 keeps the
 *   grid resident for later requests of that session with the same descriptor (< 0: a
 *   grid for this request only).  dcdz (N_el) and dvdz (N_el, may be NULL) are host
 *   arrays owned by the caller, written before tomo_server_wait returns the ticket.
 *   TOMO_ENOMEM if the request alone exceeds the budget.
 * tomo_server_submit_optimize: an optimisation request, iters (>= 1) OC iterations from
 *   the design z on the request's grid, each tomo_gradient (solves warm-started from the
 *   previous one) then tomo_oc_step with volfrac and move; the design stays on the device
 *   for the whole run and the final one is written to z_out (host, N_el, caller-owned, may
 *   be the z array) before tomo_server_wait returns.  result.compliance and result.info
 *   are those of the last gradient (the design before the last update).  Same sessions,
 *   admission and errors as tomo_server_submit (the run's four N_el buffers are added to
 *   the footprint).
 * tomo_server_wait: blocks until the ticket is done, fills *result, forgets the ticket.
 * Requests start in arrival order among those whose memory can be found (idle resident
 * grids of other sessions are evicted least recently used first, and only when that makes
 * room for the request); a request starts as soon as a worker is free, while others run.  Each request runs in order on one stream
 * on its own grid, so its result is the one it gives alone.
 * tomo_server_destroy: stops the workers after their running requests; requests still
 * queued are dropped (wait for every ticket first).
 * tomo_server_last_error: the last submit/wait error of the server, copied for the calling
 *   thread (valid until that thread's next call). */
typedef struct tomo_server tomo_server;
typedef struct {
  int64_t ticket;
  int32_t status;          /* tomo_status of the request */
  double compliance;       /* f^T u */
  tomo_solve_info info;
  double queue_ms;         /* submission to start */
  double run_ms;           /* start to completion (grid creation included when new) */
  int32_t message_len;
  char message[256];       /* error text when status != TOMO_OK */
} tomo_result;
typedef struct {
  int64_t submitted, completed, grids_created, evictions;
  uint64_t resident_bytes, peak_bytes;  /* estimated footprints of the resident grids */
  int32_t resident_grids, queued;
  int64_t batches;  /* lockstep batches run for groups of two or more gradient requests */
} tomo_server_stats;
tomo_status tomo_server_create(int32_t workers, uint64_t budget_bytes, tomo_server** out);
tomo_status tomo_server_submit(tomo_server* server, const tomo_grid_desc* desc, int64_t session,
                               const float* z, float* dcdz, float* dvdz, int64_t* ticket);
tomo_status tomo_server_submit_optimize(tomo_server* server, const tomo_grid_desc* desc,
                                        int64_t session, const float* z, int32_t iters,
                                        double volfrac, double move, float* z_out,
                                        int64_t* ticket);
tomo_status tomo_server_wait(tomo_server* server, int64_t ticket, tomo_result* result);
tomo_status tomo_server_get_stats(tomo_server* server, tomo_server_stats* stats);
/* Lockstep batching of gradient requests: with max_batch >= 2 a worker that becomes free
 * takes the first admissible request in arrival order and, when it is a gradient request,
 * every further admissible gradient request in the queue behind it, up to max_batch in
 * all, and evaluates them as one tomo_batch (lockstep CG loop, batch_workers threads and
 * streams, <= 0: 4); requests that arrive while a batch runs join the next one a worker
 * forms.  Results agree with the request alone to the solver's tolerance (tomo_batch's
 * lockstep rule); if the batch call fails, each of its requests is run alone, so one bad
 * request fails alone.  Optimisation requests always run alone.  max_batch <= 1 (the
 * default) runs every request alone on its worker's stream (bitwise the result alone).
 * Takes effect for requests a worker takes after the call. */
tomo_status tomo_server_set_batching(tomo_server* server, int32_t max_batch,
                                     int32_t batch_workers);
tomo_status tomo_server_destroy(tomo_server* server);
const char* tomo_server_last_error(const tomo_server* server);

/* Device memory held by a grid, and an upper estimate of it for a descriptor before the
 * grid exists (host staging of z, dc/dz and dV/dz included). */
tomo_status tomo_grid_device_bytes(const tomo_grid* grid, size_t* bytes);
tomo_status tomo_estimate_device_bytes(const tomo_grid_desc* desc, size_t* bytes);

/* Description of the most recent error on grid (or of the last failed tomo_create_grid
 * in this thread when grid is NULL).  Never NULL; valid until the next call on grid. */
const char* tomo_last_error(const tomo_grid* grid);

/* Host-side fault injection for tests of the error paths (no device fault is made): the
 * nth pass (>= 1) through `site` after this call fails, once, as the real call's failure
 * would: "alloc" (a device allocation of a grid: TOMO_ENOMEM), "sync" (a synchronisation
 * of a grid's stream, reported after the real one completed: TOMO_ECUDA), "graph" (the
 * launch of a captured CG loop, one grid's or a lockstep batch's: TOMO_ECUDA, nothing
 * launched), "nan_input" (a gradient's material gets one NaN modulus: the solve reports
 * TOMO_ENAN), "slow_request" (a served request waits 200 ms on the host before it runs; the
 * other workers go on).  nth = 0 disarms.  TOMO_FAULT="site:n[,site:n...]" in the environment arms
 * sites at the first check.  Process-wide; TOMO_EINVAL for an unknown site or nth < 0. */
tomo_status tomo_inject_fault(const char* site, int32_t nth);

/* Checked build (libtomo_checked.so, compiled with -DTOMO_CHECKED): the kernels' computed
 * indices are tested against their buffers' extents; the first index outside is recorded
 * (per source file) and replaced by 0, so that the access stays inside its buffer (no trap,
 * no fault; the results of that call are then wrong).  tomo_check_report synchronises the
 * device and returns *checked = 1 and in *word the first recorded violation (site in bits
 * 48-63, the index's low 48 bits below; 0: none), then clears the records.  Sites: 1/2 the
 * FP32 product's node/element loads, 3 its per-node operands (mask, b, D^-1, x_prev), 4 its
 * stores, 5 the FP64 product's loads, 6 its per-node operands, 7 the Jacobi step's moduli,
 * 8 the restriction's fine nodes and coarse moduli, 9 the prolongation's coarse nodes, 10
 * the modulus coarsening, 11 the D^-1 kernel's moduli, 12 the coarsest solve's columns, 13
 * the CG update's D^-1 gathers, 14 the filters' neighbours, 15 the sensitivity's element
 * nodes, 17 the persistent iteration's unit table, 18 the coarse tail's element, node and
 * transfer indices.  In the regular build *checked = 0 and *word = 0. */
tomo_status tomo_check_report(int32_t* checked, uint64_t* word);

#ifdef __cplusplus
}
#endif

#endif /* TOMO_H */
