/*
 * hom.h -- C ABI of the GB300 library for FFT-based homogenisation of periodic elastic cells
 * with filtered material properties (L. Gelebart and F. Ouaki, "Filtering material properties
 * to improve FFT-based methods for numerical homogenization", arXiv 1412.3228).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a):
 *   1. the per-voxel filtered stiffness c~(x_a) = HR(c, w(x_a)) of section 2: phase volume
 *      fractions inside a ball of radius r pixels around each grid point, counted on a refined
 *      grid, combined by the Voigt (eq. 3), Reuss (eq. 4) or 2-layer (eqs. 5-a, 5-b) rule;
 *   2. the basic fixed-point scheme of section 2 (eqs. 1-a, 1-b, 2): tau = (c~ - c0):eps,
 *      forward real FFT, Green operator Gamma0 on the truncated odd frequency set J with
 *      eps_hat(0) = E, inverse FFT, stress-equilibrium check -- for many cells and load cases
 *      at once;
 *   3. the effective stiffness C_eff from the volume-averaged stresses;
 *   4. the adjoint (reverse-mode) derivative of a loss on C_eff and on the local stresses.
 *
 * Conventions shared by every call
 *   - Grids have n voxels per side, n = 2^f 3^a 5^b 7^c 11^d 13^e, 3 <= n <= 2187.  The cell side is 1 and
 *     the grid points are voxel centres x_a = (a + 1/2)/n.  The paper's frequency set J is defined
 *     for odd n (section 2).  On even grids a wave vector with a Nyquist component (n/2) gets zero
 *     strain from the Green operator and is left out of the equilibrium errors.
 *   - Strains, stresses and stiffnesses use Mandel notation: 2D (plane strain) vectors hold
 *     (11, 22, sqrt2*12), nc = 3; 3D vectors hold (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12),
 *     nc = 6.  A stiffness is an nc x nc symmetric matrix stored "packed": its upper triangle
 *     row by row, ns = nc(nc+1)/2 values (6 in 2D, 21 in 3D).
 *   - Real per-voxel fields are laid out [cell][load][component][z][y][x], x fastest; cells are
 *     concatenated in the order given.  A cell's voxel offset is the sum of n^dim over the
 *     cells before it.
 *   - Every call is asynchronous on the given CUDA stream (NULL = legacy default stream) unless
 *     stated otherwise.  Pointers documented "host or device" may be either (unified
 *     addressing); pointers documented "device" must be device memory of the current device.
 *   - Caller-owned buffers are never freed by the library.  The library owns only cached FFT
 *     plans and solver workspace, which hom_release() frees.
 *   - Every function returns an int status: HOM_OK or one of the HOM_ERR_* codes below; the
 *     message of the last failure on the calling host thread is given by hom_last_error().
 *     No C++ exception crosses this interface.  The library is not re-entrant: calls that use
 *     the solver workspace must not run concurrently from several host threads.
 */
#ifndef HOM_H
#define HOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define HOM_OK 0
#define HOM_ERR_INVALID_ARG 1       /* a pointer, size or option is invalid                   */
#define HOM_ERR_UNSUPPORTED_SIZE 2  /* a prime factor above 13, n too large                      */
#define HOM_ERR_NOT_CONVERGED 3     /* some load case hit max_iter; every output is still set  */
#define HOM_ERR_DIVERGED 4          /* some load case diverged (non-finite or growing error)  */
#define HOM_ERR_TIMEOUT 5           /* a device-side wait ran out of its budget               */
#define HOM_ERR_CUDA 6              /* a CUDA runtime call failed (message has the detail)    */
#define HOM_ERR_OOM 7               /* workspace allocation failed                            */
#define HOM_ERR_CAPACITY 8          /* mixed-voxel table too small; mixed_count = needed size */
#define HOM_ERR_NOT_IMPL 9          /* requested combination is not implemented               */
#define HOM_ERR_BOUNDS 10           /* bounds-checked build (HOM_BUILD_DEBUG): a kernel found an
                                       index outside its array and skipped the access; the
                                       message names the source file id and line              */

/* ------------------------------------------------------------------ enumerations */
#define HOM_PRIM_DISK 0    /* 2D disk: centre[0..1], radius                                     */
#define HOM_PRIM_SPHERE 1  /* 3D sphere: centre[0..2], radius                                   */
#define HOM_PRIM_SLAB 2    /* slab of full thickness `radius` normal to axis `axis`, centred at */
                           /* centre[axis] (periodic)                                           */

#define HOM_RULE_NONE 0      /* c~(x_a) = c(x_a): phase of the grid point itself               */
#define HOM_RULE_VOIGT 1     /* eq. (3): sum_i f_i c_i                                          */
#define HOM_RULE_REUSS 2     /* eq. (4): (sum_i f_i c_i^-1)^-1                                  */
#define HOM_RULE_TWO_LAYER 3 /* eqs. (5-a), (5-b): two-phase laminate with the interface normal */

#define HOM_FP32 0 /* FP32 fields, FFTs and Green operator; FP64 residual norm and averages   */
#define HOM_FP64 1 /* FP64 everywhere                                                          */

#define HOM_PASSES_AUTO 0    /* specialised FP32 passes where a compiled plan exists, else generic */
#define HOM_PASSES_GENERIC 1 /* generic passes for every cell (any supported grid and precision)   */

/* Discrete Green operator (section 2, eq. 2, and the modified operators its introduction cites). */
#define HOM_GREEN_CONTINUOUS 0 /* eq. (2) at xi = 2 pi a on J (the paper's operator)                 */
#define HOM_GREEN_ROTATED 1    /* rotated finite-difference scheme: eq. (2)'s formula, and the       */
                               /* equilibrium check, at q_j = 2n sin(pi a_j/n) prod_{m!=j} cos(pi a_m/n) */

/* Iteration scheme of hom_solve (the basic scheme of section 2, or an accelerated scheme of the
 * kind its introduction and section 5 cite as complementary to filtering). */
#define HOM_SCHEME_BASIC 0       /* eqs. 1-a, 1-b, 2: eps <- E - Gamma0 * ((c~ - c0) : eps)          */
#define HOM_SCHEME_EYRE_MILTON 1 /* u = sigma + c0 : eps, u <- (I - 2 c0 Gamma0)(W u + 2 c0 : E),     */
                                 /* W = (c~ - c0)(c~ + c0)^-1: contraction (sqrt(k) - 1)/(sqrt(k) + 1) */
                                 /* for a contrast k with c0 the geometric mean of the phase moduli   */

#define HOM_CRIT_E 0  /* e   = sqrt(sum_k |xi_k . sigma_hat(k)|^2) / ||sigma_hat(0)||          */
#define HOM_CRIT_EN 1 /* e_n = sqrt(sum_{k!=0} |(xi_k/|xi_k|) . sigma_hat(k)|^2) / ||sigma_hat(0)|| */

#define HOM_STATUS_CONVERGED 0
#define HOM_STATUS_MAX_ITER 1
#define HOM_STATUS_DIVERGED 2
#define HOM_STATUS_STALLED 3   /* no new smallest error for opts->stall_window iterations       */

#define HOM_MIXED_BIT 0x80000000u /* label bit: the voxel's stiffness is in the mixed table   */

/* ------------------------------------------------------------------ inputs */

/* One analytic inclusion of a cell (cell units, periodic).  A fine-grid sample belongs to the
 * first primitive of the cell's list that contains it, else to the cell's matrix phase.
 * Disks/spheres need radius + filter radius < 1/2 of the cell; slabs need thickness < 1. */
typedef struct hom_primitive {
  int32_t kind;      /* HOM_PRIM_*                                          */
  int32_t phase;     /* index into the phase table of the call              */
  int32_t axis;      /* slab normal axis (0 = x, 1 = y, 2 = z)              */
  int32_t reserved;  /* must be 0                                           */
  double centre[3];  /* centre in cell units; centre[2] ignored in 2D       */
  double radius;     /* disk/sphere radius, or slab full thickness          */
} hom_primitive;

/* A periodic unit cell on an n^dim grid with its filter (section 2).  radius_px is the filter
 * radius in voxel units (0.5 = circle inscribed in a pixel); subgrid S is the refinement of the
 * grid on which indicator functions are averaged: the fine points are (j + 1/2)/(S n) per axis
 * and a fine point is inside the ball of voxel a when its distance to x_a is <= radius_px / n. */
typedef struct hom_cell {
  int32_t dim;          /* 2 or 3                                                 */
  int32_t n;            /* voxels per side (2^f 3^a 5^b 7^c 11^d 13^e)           */
  int32_t matrix_phase; /* phase of points outside every primitive                */
  int32_t rule;         /* HOM_RULE_*                                             */
  double radius_px;     /* filter radius in voxel units, 0 < radius_px <= (n-1)/2 */
  int32_t subgrid;      /* S, 1 <= S <= 64                                        */
  int32_t nprim;        /* number of primitives                                   */
  const hom_primitive* prims; /* host array of nprim primitives                   */
} hom_cell;

/* Isotropic phase given by its Lame constants (3D moduli; 2D cells are plane strain). */
typedef struct hom_phase {
  double lambda;
  double mu;
} hom_phase;

/* ------------------------------------------------------------------ filtered material */

/* Filtered stiffness field of a batch of cells, written by hom_filter_build into caller-owned
 * device buffers.  Each voxel has a 32-bit label: a phase index (the voxel's filter ball holds a
 * single phase, c~ = c_phase exactly), or HOM_MIXED_BIT | m where m indexes the mixed table.
 * For every mixed entry m:  c64/c32[m*ns .. m*ns+ns) packed c~ (FP64 and the same values
 * rounded to FP32), phases[2m], phases[2m+1] the two phases a < b present, frac[m] the volume
 * fraction of phase b, normal[3m..3m+3) the interface normal used by the 2-layer rule (zeros for
 * other rules), voxel[m] the global voxel index.  Mixed entries are in no particular order. */
typedef struct hom_material {
  uint32_t* label;          /* device [sum_c n_c^dim]                             */
  double* mixed_c64;        /* device [mixed_capacity * ns]                       */
  float* mixed_c32;         /* device [mixed_capacity * ns]                       */
  int32_t* mixed_phases;    /* device [mixed_capacity * 2]                        */
  double* mixed_frac;       /* device [mixed_capacity]                            */
  double* mixed_normal;     /* device [mixed_capacity * 3]                        */
  int64_t* mixed_voxel;     /* device [mixed_capacity]                            */
  int64_t mixed_capacity;   /* entries available in the mixed arrays              */
  double* phase_c64;        /* device [nphase * ns]: packed c of every phase      */
  float* phase_c32;         /* device [nphase * ns]                               */
  int32_t nphase;           /* number of phases                                   */
  int32_t dim;              /* set by hom_filter_build                            */
  int64_t mixed_count;      /* set by hom_filter_build (host-visible on return)   */
} hom_material;

/* ------------------------------------------------------------------ solver options / outputs */

typedef struct hom_solve_opts {
  int32_t precision;      /* HOM_FP32 or HOM_FP64                                       */
  int32_t criterion;      /* HOM_CRIT_E or HOM_CRIT_EN                                  */
  double tol;             /* stop when the chosen error < tol                           */
  int32_t max_iter;       /* maximum number of Green-operator applications              */
  int32_t check_every;    /* iterations launched between host polls (>= 1; 0 = default) */
  int32_t diverge_window; /* consecutive error increases that flag divergence (0 = off)  */
  int32_t use_graph;      /* 1: the whole solve as one launch of a cached CUDA graph (see  */
                          /* hom_solve); ignored when stats are requested                 */
  int32_t passes;         /* HOM_PASSES_AUTO or HOM_PASSES_GENERIC                       */
  int32_t max_radix;      /* largest register radix of the generic FP32 FFT stages: 15, 27 or
                             45 (0 = 27; FP64 always uses 15)                             */
  int32_t green;          /* HOM_GREEN_CONTINUOUS or HOM_GREEN_ROTATED (generic passes;   */
                          /* not with hom_solve_cg)                                       */
  int32_t tune;           /* 1: autotune the passes and FFT plan of FP32 solves with passes */
                          /* = AUTO and max_radix = 0, per batch shape and scheme (see     */
                          /* hom_autotune_report); 0: fixed defaults                       */
  int32_t stall_window;   /* > 0: stop a load case whose error has not reached a new minimum */
                          /* for this many iterations (HOM_STATUS_STALLED: FP32 rounding  */
                          /* floor above tol); 0 = off                                    */
  int32_t refine;         /* FP32 only: > 0 = up to this many defect corrections of the load */
                          /* cases that stall (or reach max_iter): an FP64 iteration gives  */
                          /* their error and the residual r = F(eps) - eps, and FP32       */
                          /* iterations of the correction's fixed point (source r, zero    */
                          /* mean strain) update eps in FP64.  Generic passes; the stall   */
                          /* window defaults to 30.  0 = off                               */
  int32_t refine_inner;   /* FP32 iterations per correction (0: from the FP32 iteration's */
                          /* observed contraction, enough for one correction to bring the */
                          /* error to tol / 5)                                            */
  int32_t scheme;         /* HOM_SCHEME_BASIC (0) or HOM_SCHEME_EYRE_MILTON: FP32 or FP64     */
                          /* (specialised FP32 passes in 2D), continuous Green operator,    */
                          /* hom_solve only, no refine                                      */
  int32_t warm_start;     /* 1: hom_result.eps (device, field type) holds the initial strain */
                          /* field of every load case on entry (state in / out: the returned */
                          /* fields overwrite it).  It need not be compatible: iterate 0 is */
                          /* neither checked nor returned, the first Green-operator         */
                          /* application makes it compatible with mean E.  Basic scheme of   */
                          /* hom_solve, generic passes, no refine.  0 = start from eps = E   */
} hom_solve_opts;

/* Per-kernel timing, filled when hom_result.stats is non-NULL (adds CUDA events around every
 * launch; the call then synchronises the stream before returning). */
#define HOM_NKERNEL 8
#define HOM_K_FILTER 0   /* filter build (classification, sampling, rule)                */
#define HOM_K_ROW 1      /* row pass: inverse x-FFT, constitutive, forward x-FFT          */
#define HOM_K_YFWD 2     /* 3D: forward y-FFT pass                                        */
#define HOM_K_GREEN 3    /* last-axis pass: forward FFT, Green operator, residual, inverse */
#define HOM_K_YINV 4     /* 3D: inverse y-FFT pass                                        */
#define HOM_K_CONTROL 5  /* convergence control and FP64 reductions                       */
#define HOM_K_OUTPUT 6   /* final real fields                                             */
#define HOM_K_INIT 7     /* initial state                                                 */
typedef struct hom_kernel_stats {
  int64_t launches[HOM_NKERNEL];
  double ms[HOM_NKERNEL];      /* summed CUDA-event durations of the launches              */
  double bytes[HOM_NKERNEL];   /* algorithmic HBM bytes of the work the launches performed */
  double voxel_iterations;     /* sum over (cell, load) of n^dim * iterations               */
} hom_kernel_stats;

/* Outputs of hom_solve (all caller-owned). */
typedef struct hom_result {
  void* eps;            /* optional, host or device: real strain field of the returned iterate,
                           [cell][load][nc][voxels], float (HOM_FP32) or double (HOM_FP64)   */
  void* sigma;          /* optional, same layout: stress field c~ : eps                         */
  double* mean_sigma;   /* required, host or device [ncells][L][nc]: <sigma> (FP64)            */
  int32_t* iterations;  /* optional host [ncells*L]: Green-operator applications performed     */
  int32_t* status;      /* optional host [ncells*L]: HOM_STATUS_*                              */
  double* err;          /* optional host [ncells*L]: e of the returned iterate                  */
  double* err_n;        /* optional host [ncells*L]: e_n of the returned iterate                */
  hom_kernel_stats* stats; /* optional host: per-kernel timing                                  */
  double* err_c;        /* optional host [ncells*L]: Eyre-Milton scheme only, the compatibility
                           error e_c = RMS(eps - P eps) / |E| of the returned iterate (P: the
                           projection onto compatible fields of mean E, orthogonal for c0);
                           0 for the basic scheme, whose iterates are compatible by construction */
  double* history;      /* optional, host or device [ncells*L][max_iter + 1]: entry i of a load
                           case is the stopping quantity of its iterate i (the chosen error, for the
                           Eyre-Milton scheme the larger of it and e_c; NaN for the unchecked iterate
                           0 of a warm start), written for i = 0 .. iterations (the rest untouched);
                           the FP32 iteration only when opts->refine > 0.  hom_solve only      */
} hom_result;

/* ------------------------------------------------------------------ entry points */

/* Filtered stiffness of every voxel of every cell (section 2, "Filtering mechanical
 * properties"; eqs. 3, 4, 5-a, 5-b).
 *   cells/ncells    host array of cells, all of the same dim
 *   phases/nphase   host phase table; primitives and matrices index into it
 *   mat             caller-owned outputs (see hom_material); mat->nphase must equal nphase
 *   stream          cudaStream_t or NULL
 * Volume fractions are exact sample counts on the refined grid (integer arithmetic plus a fixed
 * sequence of IEEE FP64 operations, no fused multiply-add), so they match any implementation
 * following the same recipe.  A voxel whose samples all share one phase keeps that phase's
 * stiffness exactly.  The 2-layer rule uses the normal from the centre of the primitive whose
 * surface is nearest to x_a (or the slab normal) and needs exactly two phases in the ball.
 * Synchronises the stream (the mixed-voxel count is returned in mat->mixed_count).  If the mixed
 * table is too small the labels are written, mat->mixed_count is set to the number needed and
 * HOM_ERR_CAPACITY is returned: grow the mixed arrays and call again. */
int hom_filter_build(const hom_cell* cells, int32_t ncells, const hom_phase* phases, int32_t nphase,
                     hom_material* mat, void* stream);

/* Basic fixed-point scheme (section 2, eqs. 1-a, 1-b and 2) for every cell and load case.
 *   cells/ncells  the same cells given to hom_filter_build, in the same order
 *   mat           the filtered material built for them
 *   E             host [ncells][L][nc] macroscopic strains (Mandel)
 *   L             load cases per cell (1 <= L <= 8)
 *   c0            host [ncells][2]: (lambda0, mu0) of the isotropic reference medium per cell
 *   opts          solver options
 *   out           outputs (see hom_result)
 * Per (cell, load) the iteration starts from eps = E and stops at the first iterate whose
 * equilibrium error (opts->criterion) is below opts->tol, after opts->max_iter Green-operator
 * applications, or on divergence; the returned fields and <sigma> are those of that iterate.
 * Returns HOM_OK when every load case converged, HOM_ERR_NOT_CONVERGED (max_iter or stalled) /
 * HOM_ERR_DIVERGED otherwise (all outputs still written).  Synchronises the stream before returning.
 * With opts->use_graph = 1 (and out->stats = NULL) the iterations run as one launch of a CUDA graph
 * whose conditional WHILE node repeats one iteration until the control kernel finds no active load
 * case or the iteration budget spent; the instantiated graph is kept for later calls with the same
 * arguments (same material, workspace, sizes and options; outputs may differ).
 * opts->scheme = HOM_SCHEME_EYRE_MILTON iterates u = sigma + c0 : eps instead, from u = 2 c0 : E:
 *   eps = (c~ + c0)^-1 : u per voxel (pure voxels in closed form, mixed ones through a per-call
 *   table of (c~ + c0)^-1), tau = c~ : eps - c0 : eps, and the new u_hat = tau_hat - 2 c0 :
 *   Gamma0(k) : tau_hat (k != 0; Gamma0 is left out at Nyquist bins of even grids, as in the basic
 *   scheme), u_hat(0) = tau_hat(0) + 2 c0 : E.  The iterates are not compatible before convergence,
 *   so a load case stops only when both its equilibrium error (opts->criterion) and its
 *   compatibility error e_c (hom_result.err_c) are below opts->tol.  Any positive-definite c0
 *   converges; the geometric means of the extreme phase moduli (bulk and shear) give the fastest
 *   contraction.  FP32 2D batches of specialised sizes run the specialised passes (as the basic
 *   scheme, unless opts->passes = HOM_PASSES_GENERIC), everything else the generic passes;
 *   continuous Green operator; returns HOM_ERR_NOT_IMPL with opts->green = HOM_GREEN_ROTATED or
 *   opts->refine > 0. */
int hom_solve(const hom_cell* cells, int32_t ncells, const hom_material* mat, const double* E, int32_t L,
              const double* c0, const hom_solve_opts* opts, hom_result* out, void* stream);

/* Conjugate-gradient solution of the same discrete problem as hom_solve.  The paper's introduction
 * and section 5 name Krylov schemes (its refs. [3, 12]) as complementary to filtering: they remove
 * the basic scheme's sensitivity to c0 and sharply reduce its sensitivity to the contrast.
 *   Same arguments as hom_solve without c0: the operator is eq. (2)'s Green operator for the
 *   reference medium c0 = identity (lambda0 = 0, mu0 = 1/2), G, the L2-orthogonal projection onto
 *   compatible zero-mean strain fields.  CG solves G(c~ : (E + x)) = 0 for compatible zero-mean x,
 *   with A x = G(c~ : x) symmetric positive definite.  Each step costs one row and one Green pass
 *   (the passes of hom_solve) plus five short kernels (two inner products, the updates, the control).
 *   opts->tol bounds e_G = sqrt(<r, r> / N_v) / |<sigma>| with r = -G(sigma) the projected stress of
 *   the current iterate; e_n <= e_G <= sqrt(2) e_n, so e_G is comparable to HOM_CRIT_EN (criterion
 *   is ignored, diverge_window too).  When the recursively updated residual passes, one more pass
 *   computes the true residual of E + x; the pair stops only if that passes too, else CG restarts
 *   from it.  out->err and out->err_n both receive e_G; out->iterations counts CG steps (one
 *   Green-operator application each; the start and each check add one more).
 *   HOM_STATUS_DIVERGED flags a breakdown (<p, A p> <= 0 or a non-finite value).
 *   FP32 fields reach e_G of about 6e-8 times the contrast at best (the passes round relative to the
 *   largest stress); use HOM_FP64 for contrasts of 100 and above.
 * Runs the generic passes (any supported grid, FP32 or FP64).  Synchronises the stream. */
int hom_solve_cg(const hom_cell* cells, int32_t ncells, const hom_material* mat, const double* E, int32_t L,
                 const hom_solve_opts* opts, hom_result* out, void* stream);

/* Reverse-mode derivative of a loss L(C_eff, sigma) through the fixed point (section 2, eqs. 1-a,
 * 1-b, 2) and the filter rules (eqs. 3, 4, 5-a, 5-b).  The paper does not differentiate its method;
 * this is the implicit (adjoint) derivative of the discrete problem it solves.
 *   cells, ncells, mat, c0, opts  as given to the forward hom_solve (opts->precision selects the
 *                   field type; tol / max_iter / criterion apply to the adjoint solve, whose error
 *                   is measured relative to its first residual)
 *   L               load cases per cell of the forward solve
 *   eps             device, forward strain fields [cell][load][nc][voxels] (hom_result.eps)
 *   dL_dC           host [ncells][nc][nc] dL/dC_eff, or NULL.  Needs the nc unit Mandel loads in
 *                   order (L == nc): then dC_ij/dc~(x) = eps^(i)(x) eps^(j)(x) / N_v exactly.
 *   dL_dsigma       device [cell][load][nc][voxels] dL/dsigma(x) for every voxel, or NULL.  The
 *                   adjoint field w (compatible, zero mean) solves w = -Gamma0 * ((c~-c0):w - c~:S)
 *                   and contributes (S - w) (x) eps to dL/dc~(x).
 *   dL_dctilde      device [sum voxels][ns] or NULL: dL/dc~(x), packed; entry (p <= q) is the
 *                   derivative for c~_pq and c~_qp moving together (A_pq + A_qp for p < q).
 *   dL_dphase       host [nphase][2]: dL/dlambda, dL/dmu of every phase, through the rule of every
 *                   voxel (pure voxels: c = lambda 1(x)1 + 2 mu I; mixed voxels: the rule's
 *                   forward-mode derivative).  Balls holding more than two phases are not supported.
 *   dL_dfrac        device [mat->mixed_count] or NULL: dL/df of each mixed entry (f = fraction of
 *                   its second phase, the first one taking 1 - f).
 *   adjoint_info    optional: iterations / status / err / err_n of the adjoint solves
 * Returns HOM_OK, or HOM_ERR_NOT_CONVERGED if an adjoint solve reached max_iter (outputs written).
 * Synchronises the stream. */
int hom_solve_backward(const hom_cell* cells, int32_t ncells, const hom_material* mat, const double* c0, int32_t L,
                       const hom_solve_opts* opts, const void* eps, const double* dL_dC, const void* dL_dsigma,
                       void* dL_dctilde, double* dL_dphase, double* dL_dfrac, hom_result* adjoint_info,
                       void* stream);

/* hom_solve for callers that cannot allocate device memory.  The paper has no counterpart: this is
 * a deployment variant of hom_solve, not part of the method.
 *
 * Who needs it: callers whose device memory is owned by another allocator (a framework that
 * reserved the GPU's memory up front for its caching allocator, where a foreign cudaMalloc fails
 * or fragments the pool), callers under a hard per-process memory budget, and latency-sensitive
 * callers that cannot afford the device-wide synchronisation of cudaFree.
 *
 * Same arguments, results and kernels as hom_solve (the specialised FP32 passes included), but the
 * call makes no device allocation: the FFT plan tables and all solver scratch (mixed-domain state,
 * partial sums, bookkeeping) live in one fixed array of 64 MiB in the library's device memory
 * (every device that loads the library holds it until the process exits).  A batch needing more
 * scratch than that is rejected with HOM_ERR_UNSUPPORTED_SIZE and a message giving both sizes.
 * Roughly, 2D FP32 scratch per cell is 88 * L * n * Hp bytes with Hp = (n+1)/2 rounded up to a
 * multiple of 8 (one 405^2 cell with 3 loads takes 22 MB and fits, one 1215^2 cell with 3 loads
 * takes 195 MB and does not); FP64 needs twice that, 3D cells n times more.
 *   - opts->use_graph must be 0 and out->stats must be NULL (both would allocate);
 *     HOM_ERR_INVALID_ARG otherwise.  Outputs in host memory are staged through the same array.
 *   - The basic scheme only, from eps = E: opts->scheme = HOM_SCHEME_EYRE_MILTON, opts->warm_start
 *     and opts->refine return HOM_ERR_NOT_IMPL.  A host out->history is staged through the array
 *     too (it counts towards the 64 MiB).
 *   - Every call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress); the first call on a device may load the library's device code, so
 *     make it outside any stream capture.
 *   - Every call reuses the same array and leaves its contents behind; each call re-initialises
 *     what it needs.  Calls whose GPU work overlaps (several streams or host threads at once) race
 *     on the array: serialise them.
 *   - A call that fails after queuing work waits for that work (cudaStreamSynchronize) before it
 *     returns, so its return always means that no kernel of it still uses the array.
 * Synchronises the stream before returning, like hom_solve. */
int hom_solve_noalloc(const hom_cell* cells, int32_t ncells, const hom_material* mat, const double* E, int32_t L,
                      const double* c0, const hom_solve_opts* opts, hom_result* out, void* stream);

/* Fourier extrapolation of the filtered stiffness (section 6, Fig. 4): the truncated Fourier series
 * of one component of c~ whose coefficients are the DFT of its grid values x_a = (a + 1/2)/n on the
 * odd frequency set J, evaluated at the voxel centres y_b = (b + 1/2)/m of a finer m^dim grid:
 *     f(y) = n^-dim sum_{k in J} c_hat(k) exp(2 pi i k.(y - x_0)),   x_0 = 1/(2n) per axis,
 * which reproduces c~(x_a) wherever a fine point coincides with a grid point.  A diagnostic of how
 * the spectral method "sees" the filtered microstructure between grid points.  Computed in FP64.
 *   cells/ncells  the batch given to hom_filter_build, mat its material
 *   cell          index of the cell to extrapolate
 *   comp          packed component of c~ (upper triangle row by row: 0 = c~_11, 1 = c~_12, ...)
 *   (odd grids only: J is symmetric there, so the series is real)
 *   m             fine points per side, 1 <= m <= 32768 in 2D, <= 1024 in 3D (m < n samples the
 *                 series more coarsely than the grid; m = n returns c~(x_a) itself)
 *   out           host or device [(m,) m, m] float64, x fastest; caller-owned
 *   stream        cudaStream_t or NULL
 * Allocates scratch of about n^dim + n m^(dim-1) doubles (plus m^dim when out is host memory) on
 * the stream; HOM_ERR_OOM if that fails.  Synchronises the stream. */
int hom_fourier_extrapolate(const hom_cell* cells, int32_t ncells, const hom_material* mat, int32_t cell,
                            int32_t comp, int32_t m, double* out, void* stream);

/* Effective stiffness from mean stresses: <sigma^(l)> = C_eff E^(l) for the L = nc linearly
 * independent load cases of each cell, so C_eff = S^T (E^T)^-1 (with the nc unit Mandel strains
 * as loads, column l of C_eff is <sigma^(l)>).  Computed in FP64 on the host.
 *   ncells, dim   batch description
 *   E             host [ncells][nc][nc] load cases (row l = E^(l))
 *   mean_sigma    host or device [ncells][nc][nc] (row l = <sigma^(l)>, as hom_solve writes)
 *   C_out         host [ncells][nc][nc] row-major
 * Returns HOM_ERR_INVALID_ARG if some E is singular.  Synchronous. */
int hom_effective_stiffness(int32_t ncells, int32_t dim, const double* E, const double* mean_sigma,
                            double* C_out);

/* The autotuner's record.  The first FP32 hom_solve of a batch shape (device, dimension, load count,
 * Green operator, multiset of grid sizes) with opts->tune = 1 (passes = AUTO, max_radix = 0) times
 * four candidate plans on that batch -- the specialised passes and the generic passes with register
 * radices up to 15, 27 and 45 -- over 4 fixed iterations each (after one untimed call), and every
 * later solve of the shape runs the fastest.  Writes one line per shape, "shape: timings -> choice",
 * into buf (at most len bytes, NUL-terminated) and returns the full length.  The choice depends on
 * measured times, so two processes may pick different plans (results then differ by FP32 rounding). */
int32_t hom_autotune_report(char* buf, int32_t len);

/* Message of the last failed call on this host thread ("" if none). */
const char* hom_last_error(void);

/* Frees cached FFT plans and solver workspace on every device the library used. */
void hom_release(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t hom_version(void);

/* Build flags of the loaded library: HOM_BUILD_DEBUG when it was compiled with -DHOM_DEBUG, whose
 * solver kernels check their global indices (state, g, output fields, labels) and their task
 * descriptors against the arrays' extents, record the first failure and skip the access (the call
 * then returns HOM_ERR_BOUNDS), and fill their dynamic shared memory with NaN bytes before use. */
#define HOM_BUILD_DEBUG 1
int32_t hom_build_flags(void);

#ifdef __cplusplus
}
#endif

#endif /* HOM_H */
