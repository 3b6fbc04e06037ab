/*
 * cpm.h -- C ABI of libcpm: the GB300 (sm_103a) hot path of the closest point
 * method (CPM) solver for the shifted surface Poisson problem
 *
 *     (c - Delta_S) u = f                                   (Section 1, eq. shiftPoisson)
 *
 * of May, Haynes & Ruuth, "A closest point method library for PDEs on surfaces
 * with parallel domain decomposition solvers and preconditioners" (arXiv
 * 2110.06322), discretised on a narrow band of a uniform grid (Section 2.1)
 * and solved by GMRES preconditioned by restricted additive Schwarz with
 * Dirichlet (RAS) or Robin (ORAS) transmission (Section 2.2, Section 4.1.1).
 *
 * Conventions shared by every call
 *   - Vectors are CALLER-OWNED DEVICE pointers of length N_A (the number of
 *     active band nodes), in the band's canonical order: lexicographic in the
 *     lattice index (i, j, k), k fastest.  Lattice node (i, j, k) is the point
 *     (i h, j h, k h).  Several right-hand sides are stored one after another
 *     (rhs-major, N_A apart).
 *   - Handles (cpm_band, oras_pc) are LIBRARY-OWNED; free them with the
 *     matching *_free call.  They live on the device that was current when
 *     they were built.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     is ordered on it.  Only cpm_band_build, oras_setup and cpm_solve* wait
 *     on the host (to size allocations and to fill the info struct).
 *   - Working memory comes stream-ordered from the device's default memory
 *     pool (cudaMallocAsync).  On its first allocation on a device the library
 *     raises that pool's release threshold to 64 GiB, so that memory freed by
 *     one solve or set-up is reused by the next instead of being unmapped at
 *     every synchronisation; cudaMemPoolTrimTo on the default pool gives it
 *     back.
 *   - Errors are returned as cpm_status codes; a message for the last error
 *     of the calling thread is available from cpm_last_error().  No call
 *     aborts the process or traps the device.  Kernels that wait on a
 *     condition bound their wait and report CPM_ERR_TIMEOUT.
 */
#ifndef CPM_H
#define CPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CPM_OK = 0,
  CPM_ERR_ARG = 1,            /* invalid argument (null pointer, size, kind) */
  CPM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  CPM_ERR_OOM = 3,            /* device allocation failed */
  CPM_ERR_BAND = 4,           /* band not within the surface reach, or not closed */
  CPM_ERR_NOT_CONVERGED = 5,  /* iteration limit reached before the tolerance */
  CPM_ERR_BREAKDOWN = 6,      /* zero pivot in ILU(0) or Krylov breakdown */
  CPM_ERR_NAN = 7,            /* NaN or Inf met in an input or a residual */
  CPM_ERR_TIMEOUT = 8         /* a bounded device-side wait ran out */
} cpm_status;

typedef enum { CPM_F64 = 0, CPM_F32 = 1, CPM_BF16 = 2 } cpm_dtype;

/* Surface (Section 2.1, closest point function eq. cpFunc).
 *   kind 0: sphere,  param = {cx, cy, cz, rho}
 *   kind 1: torus about the z axis through (cx, cy, cz), param = {cx, cy, cz, R, r}, R > r > 0 */
typedef struct {
  int32_t kind;
  double param[8];
} cpm_surface;

typedef struct cpm_band cpm_band;
typedef struct oras_pc oras_pc;

/* ------------------------------------------------------------------ band
 * cpm_band_build -- build the computational band (Section 2.1): the seed tube
 * T = {x : dist(x, S) <= lambda}, lambda = h sqrt(2((p+1)/2)^2 + (1+(p+1)/2)^2)
 * (sqrt(17) h for p = 3); the active set Sigma_A = union over x in T of the
 * (p+1)^3 interpolation cube at cp(x), with base b = floor(cp/h - (p-1)/2);
 * the ghost set Sigma_G = 6-neighbours of Sigma_A outside it; and one
 * extension (E) row per node of Sigma_A and Sigma_G.
 *   surf   host pointer to the surface;  h > 0;  p in {2, 3}.
 *   out    receives the new handle (library-owned).
 * Returns CPM_ERR_BAND when lambda >= the reach kappa^-1 (sphere rho, torus
 * min(r, R - r)) or when some E-row cube leaves Sigma_A. */
cpm_status cpm_band_build(const cpm_surface* surf, double h, int p, void* stream, cpm_band** out);
/* (cpm_band_build also commits, once per device, the fixed scratch array of
 * cpm_apply_noalloc below.) */

/* Sizes of the band: |Sigma_A|, |Sigma_G|, |T|. Host pointers; any may be NULL. */
cpm_status cpm_band_info(const cpm_band* band, int64_t* n_active, int64_t* n_ghost, int64_t* n_tube);

/* Export the band to caller-owned DEVICE buffers (any may be NULL):
 *   ijk_active [N_A x 3] int32, canonical order
 *   ijk_ghost  [N_G x 3] int32, canonical order
 *   erow_base  [N_C x 3] int32 and erow_cp [N_C x 3] double, N_C = N_A + N_G,
 *              rows of Sigma_A (canonical) followed by rows of Sigma_G (canonical)
 *   perm       [N_A] int64: position of canonical node q in the library's vectors
 *              (the identity: vectors are stored in canonical order). */
cpm_status cpm_band_export(const cpm_band* band, int32_t* ijk_active, int32_t* ijk_ghost, int32_t* erow_base,
                           double* erow_cp, int64_t* perm, void* stream);

/* Export the 1-D barycentric interpolation weights of every E row (Section
 * 2.1, tensor-product barycentric Lagrange interpolation of degree p) to a
 * caller-owned DEVICE buffer w1d [N_C x 3 x (p+1)] double, rows ordered as in
 * cpm_band_export.  The tensor weight of cube node (u, v, w) is
 * (w1d[r][0][u] * w1d[r][1][v]) * w1d[r][2][w]. */
cpm_status cpm_band_weights(const cpm_band* band, double* w1d, void* stream);

/* ------------------------------------------------------------------ operator
 * cpm_apply -- y = M x (transpose = 0) or y = M^T x (transpose = 1), with
 *   M = c I - Delta_S^h,  Delta_S^h = -(2d/h^2) I + (Delta^h + (2d/h^2) I) E
 * (Section 2.1, eq. lapBel; d = 3): y_i = (c + 6/h^2) x_i - (1/h^2) sum over
 * the six neighbours n of i of (E x)_n.  Matrix-free: each E row gathers its
 * (p+1)^3 cube.
 *   c      HOST array of nrhs shifts (c > 0 in the paper; any finite value accepted)
 *   x, y   DEVICE buffers of nrhs x N_A elements of `dtype` (CPM_F64 or CPM_F32);
 *          x and y must not overlap.
 * The transposed apply gathers E^T through a precomputed transpose map (no
 * atomics, deterministic). */
cpm_status cpm_apply(const cpm_band* band, const double* c, const void* x, void* y, cpm_dtype dtype, int nrhs,
                     int transpose, void* stream);

/* cpm_apply_noalloc -- the forward operator of cpm_apply (y = M x, same
 * arguments and layout, no transpose) for callers that cannot allocate device
 * memory: processes whose device memory belongs to another allocator (a
 * framework's caching pool that has reserved the device) or latency-bounded
 * loops in which an allocation may block.  This is not an operation of the
 * paper; it only changes where the apply's scratch comes from.
 *   Scratch: one fixed 16 MiB array inside the library.  It is committed on a
 *   device when the first band is built there (cpm_band_build looks up the
 *   array's device address with that device current, which under CUDA's lazy
 *   module loading is what loads it) and held until the process exits, so a
 *   caller that builds its bands before handing the device to another
 *   allocator needs no allocation later.  A call needs
 *   min(nrhs, 16) x N_C x 8 bytes (N_C = N_A + N_G); larger calls are rejected
 *   with CPM_ERR_ARG and a message naming the sizes.  More than 16 right-hand
 *   sides run 16 at a time through the same scratch.
 *   All calls share the array: calls whose kernels overlap on the GPU race.
 *   Allocates nothing (no cudaMalloc, no stream-ordered or library allocation;
 *   cpm_device_allocations() does not change). */
cpm_status cpm_apply_noalloc(const cpm_band* band, const double* c, const void* x, void* y, cpm_dtype dtype,
                             int nrhs, void* stream);

/* ------------------------------------------------------------------ Schwarz preconditioner
 * (Section 2.2; defaults of Section 4.1.1: alpha = 4, alpha_cross = 20, ILU(0) local solves)
 *   nparts       number of disjoint subdomains N_S, from recursive coordinate
 *                bisection of Sigma_A by lattice planes; an overlapping
 *                subdomain may hold at most 65,535 rows (the packed factors
 *                carry 16-bit local columns): oras_setup returns CPM_ERR_ARG
 *                beyond that, and a larger nparts is the remedy
 *   overlap      N_O: layers of 6-adjacency within Sigma_A added to each part
 *   robin        0: RAS (Dirichlet transmission); 1: ORAS with the Robin reading
 *                A_j[i,i] += D_i / (1 + alpha h), D_i the sum of the entries of
 *                row i of M dropped by the restriction (alpha_cross when those
 *                columns belong to two or more other parts)
 *   store        precision of the stored factors used by oras_apply with
 *                CPM_F32 vectors: CPM_F32 or CPM_BF16 (FP64 factors are always kept) */
typedef struct {
  int32_t nparts;
  int32_t overlap;
  int32_t robin;
  double alpha;
  double alpha_cross;
  int32_t store;
  int32_t order;  /* local order of the ILU(0) factorisation: 1 descending distance
                     to the surface; 2 distance shells of width h (outermost
                     first), then lattice-parity colours; ties canonical;
                     0 by degree: 2 for p = 3 (fewer GMRES iterations and
                     shallower sweeps), 1 for p = 2 (where the shell order
                     costs iterations) */
  int32_t coarse; /* 0 one-level (the paper's preconditioners); 1 two-level:
                     a coarse correction on the space Z of one constant per
                     disjoint part, E0 = Z^T M Z, applied before the
                     one-level apply: q = Z E0^{-1} Z^T r,
                     z = q + P_1(r - M q) (transposed: t = P_1^T r,
                     z = t + Z E0^{-T} Z^T (r - M^T t)).  The paper names a
                     coarse grid correction as future work (Section 4.1.1);
                     this is the reading built here. */
} oras_params;

/* oras_setup -- partition, overlap growth, local matrices A_j = R_j M R_j^T
 * (+ Robin term), and ILU(0) of each A_j in its local order (prm->order: 1
 * descending distance to the surface, ties by canonical index; 2 distance
 * shells of width h, then lattice-parity colours; 0 chosen by the degree p).
 * c is the shift of M.
 * The paper leaves the local order to PETSc (Section 4.1.1). */
cpm_status oras_setup(const cpm_band* band, const oras_params* prm, double c, void* stream, oras_pc** out);

/* oras_apply -- z = sum_j Rtilde_j^T (L_j U_j)^{-1} R_j r (transpose = 0) or
 * z = sum_j R_j^T (L_j U_j)^{-T} Rtilde_j r (transpose = 1): restrict to the
 * overlapping subdomains, solve with the ILU(0) factors, and keep each
 * subdomain's values on its own disjoint part.  r, z: DEVICE, nrhs x N_A of
 * dtype (CPM_F64 or CPM_F32), not overlapping. */
cpm_status oras_apply(const oras_pc* pc, const void* r, void* z, cpm_dtype dtype, int nrhs, int transpose,
                      void* stream);

/* Run-time settings of a preconditioner's apply.  None changes the result of
 * a successful apply beyond the summation order inside a row; they choose
 * among equivalent kernels and exercise the failure path.  The paper has no
 * counterpart (its subdomain solves are PETSc calls, Section 4.1.1).
 *   xplace         where each subdomain's local vector lives during the
 *                  triangular sweeps: 0 in shared memory when it fits beside the
 *                  factor ring (default), else in a global-memory slice; 1
 *                  always in a global-memory slice; 2 (FP32 applies) as 0, but
 *                  where the FP32 local vector does not fit it is held in FP16
 *                  in shared memory (one CTA per SM, 8 lanes per row, 12
 *                  consumer warps) when that fits: the entries of R_j r are
 *                  scaled by a power of two per subdomain so the largest is
 *                  in [1, 2), and rows that carry a reciprocal pivot are
 *                  computed as (x_i sigma - sum) / pivot with sigma the power
 *                  of two at the binade of c + 6/h^2 (the pivots lie within a
 *                  small factor of it), so stored values stay in FP16's normal
 *                  range; arithmetic stays FP32.  This changes the
 *                  preconditioner's rounding (about 1e-3 relative), not the
 *                  method; the FP32 inner cycles of the mixed solver are
 *                  flexible, so they use exactly the preconditioned vectors
 *                  they computed.  3 as 2 with 24 consumer warps.  FP64
 *                  applies treat 2 and 3 as 0.  The autotuner tries 0 and 1 only.
 *   lanes          lanes of a warp per factor row in the sweeps: 4, 8 or 16
 *                  (0: 8)
 *   schedule       order in which subdomains are handed to CTAs: 0 longest
 *                  first (default), 1 partition order
 *   ctas           CTAs per SM when the local vectors live in global slices: 1
 *                  one, with a 64 KB shared-memory carve-out that leaves the rest
 *                  of the SM's 256 KB to the L1 cache holding the slice (0: the
 *                  default, this one); 2 two; 4 four, of 6 consumer warps each
 *                  (8 lanes per row), so that up to 608 subdomains run at once
 *   probe_timeout  0 normal; 1 failure-path test: the first factor-chunk wait
 *                  of every subdomain waits on a barrier that nothing completes,
 *                  so each CTA runs out after wait_polls polls, waits for its
 *                  copies in flight and returns; the next cpm_solve reports
 *                  CPM_ERR_TIMEOUT (the GPU context stays usable)
 *   wait_polls     polls of each consumer-side bounded wait before it gives up
 *                  (0: the default, 2^22 polls, seconds at most)
 * pc: library-owned handle; t: HOST pointer.  Not stream-ordered: set it
 * while no apply of pc is running. */
typedef struct {
  int32_t xplace;
  int32_t lanes;
  int32_t schedule;
  int32_t ctas;
  int32_t probe_timeout;
  int64_t wait_polls;
} oras_tuning;
cpm_status oras_set_tuning(oras_pc* pc, const oras_tuning* t);
cpm_status oras_get_tuning(const oras_pc* pc, oras_tuning* t);

/* oras_autotune -- time every combination of xplace (both when the local
 * vectors fit in shared memory), lanes (4, 8, 16), schedule (0, 1) and ctas
 * (1, 2, 4; where the local vectors live in global slices) on
 * `reps` forward applies of dtype (CPM_F32 or CPM_F64) each, with CUDA events
 * on `stream`, and keep the fastest as the preconditioner's setting (the
 * probe stays off).  best (HOST, may be NULL) receives it and best_ms (HOST,
 * may be NULL) its time per apply.  Allocates two vectors of N_A values for
 * the duration of the call; synchronises the stream. */
cpm_status oras_autotune(oras_pc* pc, cpm_dtype dtype, int reps, void* stream, oras_tuning* best, double* best_ms);

/* Sizes of the preconditioner: number of parts, sum of |S_j|, sum of nnz(A_j),
 * and the largest number of forward-solve levels of any subdomain.  Host pointers. */
cpm_status oras_info(const oras_pc* pc, int32_t* nparts, int64_t* total_rows, int64_t* total_nnz,
                     int32_t* max_levels);

/* Export the disjoint partition part[N_A] (int32) and the overlapping
 * subdomains, concatenated in local order (int32 canonical node indices),
 * with offsets sub_ptr[nparts + 1] (int64).  DEVICE buffers; any may be NULL. */
cpm_status oras_export(const oras_pc* pc, int32_t* part, int64_t* sub_ptr, int32_t* sub_nodes, void* stream);

/* ------------------------------------------------------------------ solver
 * Restarted GMRES(restart), right preconditioned by the Schwarz preconditioner
 * (Section 4.1.1: GMRES is the default Krylov method): classical Gram-Schmidt
 * (reorth 0: one pass, the refinement-free classical Gram-Schmidt of PETSc's
 * GMRES, on which the paper's solver is built (Section 1); 1: a second pass when
 * the first shrank the vector below 1/sqrt(2) of its norm; 2: always two
 * passes), Givens least squares, stop
 * when |f - M u|_2 <= rtol |f|_2 (true residual, FP64).
 * mixed = 1: FP64 iterative refinement around an inner GMRES whose operator
 * and preconditioner applies run in FP32 (factors stored per oras_params.store);
 * the outer residual, Gram-Schmidt and the least-squares update stay FP64. */
typedef struct {
  int32_t restart;
  int32_t maxit;      /* total inner GMRES iterations allowed */
  double rtol;
  int32_t mixed;
  int32_t reorth;
  double inner_rtol;  /* mixed only: relative tolerance of each inner solve */
  int32_t timing;     /* 1: time the preconditioner and operator applies with CUDA
                         events on `stream` (adds one event wait per apply) */
} cpm_solve_params;

typedef struct {
  int32_t iters;         /* GMRES iterations (inner iterations summed when mixed) */
  int32_t restarts;      /* GMRES cycles */
  int32_t ir_steps;      /* refinement steps (mixed) */
  double rel_residual;   /* |f - M u|_2 / |f|_2 in FP64 at exit */
  int32_t status;        /* cpm_status of the solve */
  double ms_precond;     /* timing = 1: total milliseconds in preconditioner applies */
  double ms_operator;    /* timing = 1: total milliseconds in operator applies */
  int32_t n_precond;     /* number of preconditioner applies */
  int32_t n_operator;    /* number of operator applies */
} cpm_solve_info;

/* cpm_solve -- solve M u = f.  f: DEVICE, N_A doubles.  u: DEVICE, N_A
 * doubles, initial guess on entry, solution on exit.  pc may be NULL (no
 * preconditioner).  info: HOST.  Synchronises the stream. */
cpm_status cpm_solve(const cpm_band* band, const oras_pc* pc, double c, const double* f, double* u,
                     const cpm_solve_params* prm, cpm_solve_info* info, void* stream);

/* cpm_solve_adjoint -- solve M^T lambda = g with the transposed operator and
 * the transposed preconditioner (same conventions as cpm_solve). */
cpm_status cpm_solve_adjoint(const cpm_band* band, const oras_pc* pc, double c, const double* g, double* lambda,
                             const cpm_solve_params* prm, cpm_solve_info* info, void* stream);

/* cpm_solve_batch -- solve many independent systems in lockstep: problem p
 * (p < nprob) has its own band, preconditioner pcs[p] (NULL: none; pcs may
 * be NULL for none anywhere) and shift c[p] (HOST array), and nrhs[p] >= 1
 * right-hand sides, each solved with the same GMRES(restart) as cpm_solve
 * (one classical Gram-Schmidt pass; prm->reorth is not used).
 *   f, u   DEVICE, the concatenation over p of nrhs[p] x N_A(p) doubles
 *          (problem-major, right-hand side within problem); u holds the
 *          initial guesses on entry and the solutions on exit.
 *   info   HOST array of sum(nrhs) entries, one per system in that order.
 *   transpose  1: solve the adjoint systems M^T u = f.
 * Every iteration applies the operator and the preconditioner once per
 * problem for all its right-hand sides; the Krylov vector work runs over the
 * whole batch in single launches with per-system reductions.  A system stops
 * on the device when its residual estimate reaches rtol |f| and is frozen
 * until the others finish their cycle; each cycle ends with every system's
 * true FP64 residual.  mixed = 1 runs the operator and preconditioner in FP32
 * inside FP64 iterative refinement (FP32 or BF16 factors required), each
 * inner cycle flexible (the correction is sum_j y_j P v_j over the kept
 * preconditioned vectors).
 * The lockstep solver keeps (restart + 7) doubles per unknown of every system
 * it runs at once (2 restart + 7 with mixed = 1), so the problems are cut, in order, into consecutive
 * groups whose storage fits min(32 GB, 40 % of the device's free memory),
 * solved one group after another within the call.
 * Returns CPM_ERR_NOT_CONVERGED if any system missed rtol within maxit
 * iterations (its info[] entry says which).  Synchronises the stream.
 * The paper solves one problem per PETSc run; batching is this library's. */
cpm_status cpm_solve_batch(int32_t nprob, const cpm_band* const* bands, const oras_pc* const* pcs, const double* c,
                           const int32_t* nrhs, const double* f, double* u, const cpm_solve_params* prm,
                           cpm_solve_info* info, int32_t transpose, void* stream);

/* ------------------------------------------------------------------ reaction-diffusion (IMEX)
 * Schnakenberg system of eq. schnack (Section 4.1.6) on the band,
 *   u_t = D_u Delta_S u + delta1 - u + u^2 v + lambda v
 *   v_t = D_v Delta_S v + delta2 - u^2 v - lambda v,
 * advanced by semi-implicit Euler steps (diffusion implicit, reaction
 * explicit): each step solves (c_u I - Delta_S^h) u' = c_u (u + dt f(u, v))
 * with c_u = 1 / (D_u dt), and the same for v -- two shifted Poisson solves
 * (cpm_solve with c = c_u, c_v).  The paper's reaction-diffusion examples
 * treat diffusion implicitly with PETSc's IMEX Runge-Kutta schemes (Section
 * 4.1.3, Section 4.1.5); the step here is the first-order member of that
 * family. */
typedef struct {
  double delta1, delta2, lambda;  /* reaction parameters (eq. schnack) */
  double Du, Dv;                  /* diffusion coefficients, > 0 */
  double dt;                      /* step, > 0 */
  int32_t model;                  /* 0 the Schnakenberg reaction; 1 no reaction: each
                                     species follows the heat equation u_t = D Delta_S u
                                     (Section 4.1.3) */
} cpm_schnakenberg;

/* cpm_imex_rhs -- right-hand sides of one step:
 *   bu = c_u (u + dt f(u, v)),  bv = c_v (v + dt g(u, v)).
 * u, v, bu, bv: DEVICE, N_A doubles each (bu, bv must not overlap u, v). */
cpm_status cpm_imex_rhs(const cpm_band* band, const cpm_schnakenberg* prm, const double* u, const double* v,
                        double* bu, double* bv, void* stream);

/* cpm_imex_rhs_adjoint -- reverse of one step for a loss L of the state after it.
 *   u, v     state before the step;  u1, v1 state after it (DEVICE, N_A each)
 *   lu, lv   adjoint solutions M_u^{-T} dL/du1, M_v^{-T} dL/dv1 (DEVICE)
 *   ubar     = dL/du through this step = c_u lu (1 + dt f_u) + c_v lv dt g_u
 *   vbar     = dL/dv through this step = c_u lu dt f_v + c_v lv (1 + dt g_v)
 *   dc       DEVICE, 2 doubles, ACCUMULATED: dc[0] += <lu, u + dt f - u1> and
 *            dc[1] += <lv, v + dt g - v1>, this step's dL/dc_u and dL/dc_v
 *            (over all steps, dL/dD_u = -(c_u / D_u) dc[0]).
 * The sums use a fixed reduction order (reproducible). */
cpm_status cpm_imex_rhs_adjoint(const cpm_band* band, const cpm_schnakenberg* prm, const double* u, const double* v,
                                const double* u1, const double* v1, const double* lu, const double* lv,
                                double* ubar, double* vbar, double* dc, void* stream);

/* cpm_imex2_rhs -- right-hand sides of the two implicit stages of one
 * second-order IMEX Runge-Kutta step, ARS(2,2,2) (Ascher, Ruuth & Spiteri
 * 1997; the paper's reaction-diffusion and heat examples use PETSc's IMEX
 * Runge-Kutta schemes, Section 4.1.3 and Section 4.1.5).  With
 * gamma = 1 - 1/sqrt(2), delta = 1 - 1/(2 gamma), F = (f, g) the reaction and
 * the shifts c_u = 1 / (gamma D_u dt), c_v = 1 / (gamma D_v dt), each stage
 * solves M(c) U = b (cpm_solve with c = c_u, c_v):
 *   stage 2:  bu = c_u (u + gamma dt f(u, v))
 *   stage 3:  bu = c_u (u + dt (delta f(u, v) + (1 - delta) f(u2, v2))
 *                      + ((1 - gamma) / gamma) (u2 - u - gamma dt f(u, v)))
 * and likewise bv; the step's result is the stage-3 solution.
 *   u, v     state at the start of the step; u2, v2 the stage-2 solutions
 *            (stage 3 only; may be NULL for stage 2)
 * All DEVICE, N_A doubles; bu, bv must not overlap the inputs. */
cpm_status cpm_imex2_rhs(const cpm_band* band, const cpm_schnakenberg* prm, int32_t stage, const double* u,
                         const double* v, const double* u2, const double* v2, double* bu, double* bv, void* stream);

/* cpm_dot -- out[0] = <a, b> over N_A doubles (DEVICE a, b, out), in a fixed
 * reduction order.  Used by gradients with respect to the shift c
 * (dL/dc = -<lambda, u> for u = M^{-1} f). */
cpm_status cpm_dot(const cpm_band* band, const double* a, const double* b, double* out, void* stream);

void cpm_band_free(cpm_band* band);
void oras_free(oras_pc* pc);

/* Total number of CUDA kernels this library has launched since it was loaded
 * (all threads).  The difference of two readings counts the kernels of the
 * calls made in between. */
int64_t cpm_kernel_launches(void);

/* Total number of device allocations (stream-ordered cudaMallocAsync calls)
 * this library has made since it was loaded (all threads).  The difference of
 * two readings counts the allocations of the calls made in between. */
int64_t cpm_device_allocations(void);

/* Message of the last failed call on this thread ("" if none). */
const char* cpm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CPM_H */
