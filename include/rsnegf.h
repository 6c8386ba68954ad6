/*
 * rsnegf.h -- C ABI of the GB300 (sm_103a) real-space NEGF transmission library.
 *
 * The library computes, on one GPU, the Landauer transmission of a junction
 * described on a real-space grid with absorbing boundary conditions
 * (Feldman, Seideman, Hod & Kronik, "A real-space method for highly
 * parallelizable electronic transport calculations"):
 *
 *   H_op   = H_KS - i Gamma,  Gamma = Gamma_L + Gamma_R          (Sec. II.B, Eq. Hop)
 *   G^r(E) = (E 1 - H_op)^{-1} = (E - H_KS + i Gamma)^{-1}        (Sec. II.A, Eq. G)
 *   T(E)   = 4 sum_{i in L, j in R} Gamma_L,i Gamma_R,j |G_ij|^2  (Sec. II.B, Eq. T-realspace;
 *            the factor 4 is the coupling Gamma_std = 2*CAP, since the CAP is the
 *            anti-Hermitian part of the lead self-energy)
 *
 * H_KS is real symmetric: -1/2 times an order-2R finite-difference Laplacian,
 * a local potential V_loc and separable Kleinman-Bylander projectors
 * (Sec. II.C: the only off-diagonal entries are the FD stencil and the
 * cutoff-limited nonlocal part).  Because H_op is complex symmetric
 * (Eq. complex-sym) G = G^T, so T needs only the columns x_j = G e_j for the
 * grid points j with Gamma_R,j > 0.  Each column is found by a Krylov solve of
 * A(E) x_j = e_j (conjugate orthogonal conjugate gradients, COCG -- the paper
 * itself diagonalises instead; the column solve is this library's route),
 * with iterative refinement on the true residual in FP64.
 *
 * Conventions for every entry point:
 *  - Grid: nx*ny*nz points, flat index ix + nx*(iy + ny*iz) (x fastest),
 *    spacing h (bohr), zero (Dirichlet) values outside the box on every axis.
 *    Transport axis z.  Energies in hartree.
 *  - Complex vectors are interleaved (re, im): complex128 = two doubles,
 *    complex64 = two floats.
 *  - Pointers named *_dev are device pointers (cudaMalloc / PyTorch memory on
 *    the context's device); every other pointer is host memory.  The caller owns
 *    all buffers it passes; setters copy their inputs, so host arrays may be
 *    freed after the call returns.
 *  - Work is queued on the context's stream.  Calls that return host results
 *    (T, dV, iteration counts) synchronise that stream before returning; calls
 *    that only write *_dev buffers may return before the GPU is done.
 *  - Every call returns an rsn_status and never aborts the process; on failure
 *    rsn_last_error() describes the cause.  A context is used by one host
 *    thread at a time.
 */
#ifndef RSNEGF_H
#define RSNEGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsn_ctx rsn_ctx; /* opaque: device copies of the setup data, workspaces, graphs */

typedef enum {
    RSN_OK = 0,
    RSN_EINVAL = -1,     /* bad argument (null pointer, size, range, call order) */
    RSN_ENOMEM = -2,     /* device or host allocation failed */
    RSN_ECUDA = -3,      /* a CUDA runtime call failed (no device, launch error, ...) */
    RSN_ENOCONV = -4,    /* some columns missed the tolerance within max_outer sweeps */
    RSN_ETIMEOUT = -5,   /* deadline_ms elapsed before every column converged */
    RSN_EBREAKDOWN = -6, /* COCG breakdown (p^T A p ~ 0) persisted across restarts */
    RSN_ESTATE = -7      /* required setter not called yet */
} rsn_status;

enum { RSN_FP64 = 0, RSN_MIXED = 1 };

/* Solver options (rsn_default_opts fills every field). */
typedef struct {
    int precision;      /* RSN_FP64: complex FP64 Krylov recurrence;
                           RSN_MIXED: complex FP32 recurrence on the correction
                           equation, FP64 true residual / update / T sums. */
    double tol;         /* stop when ||b - A x||_2 <= tol * ||b||_2 (true residual, FP64) */
    double tol_inner;   /* reliable-update factor (0 < tol_inner < 1): once the recurrence
                           residual has dropped by this factor since the last true residual,
                           the FP64 true residual b - A x replaces it (the search direction is
                           kept) or, if below tol, finishes the system */
    int max_iter;       /* cap on Krylov iterations per system */
    int max_outer;      /* cap on true-residual replacements per system */
    double deadline_ms; /* wall-clock budget of the call, 0 = none */
    int rhs_block;      /* slots: systems solved concurrently (0 = automatic); the
                           remaining systems wait in a queue and take freed slots */
    int use_graph;      /* 1: replay the iteration body as a captured CUDA graph */
    int graph_iters;    /* iterations per graph replay between convergence polls (1..256) */
    int timing;         /* 1: time every COCG operator / update launch with CUDA events
                           (read back with rsn_kernel_stats) */
    double tol_adjoint; /* tolerance of the adjoint systems of rsn_transmission_vjp (0 = tol).
                           Their right-hand side Gamma_L o conj(x_j) is built from a computed
                           column, and on large, nearly resonant junctions the FP64 recurrence
                           of an adjoint can level off above a tol that its forward column
                           meets; a looser target here keeps tol for the columns and T */
    double tol_T;       /* goal-oriented finish of the forward columns (b = e_j): once the
                           true residual meets tol, iterations continue until
                           t_j = sum_{i in L} Gamma_L,i |x_j(i)|^2 -- the column's share of
                           Eq. T-realspace -- changes by at most tol_T * t_j between two true
                           residuals.  Where every lead channel is closed, x_j is exponentially
                           small on the Gamma_L support and a residual of tol relative to the
                           whole column fixes t_j only to ~1e-3 (tol 1e-10) or ~1e-6 (1e-13);
                           the iterate keeps converging there after its residual reaches the
                           rounding floor.  Measured on the 24x24x120 junction against the
                           oracle's LU: tol_T 1e-7 (mixed default) leaves T within ~1e-7 and
                           each t_j within ~1e-4 (the tiniest shares); 3e-11 (FP64 default)
                           within ~1e-10.
                           0 = residual criterion alone. */
} rsn_solver_opts;

/* Defaults for a precision: FP64 -> tol 1e-13, tol_T 3e-11, tol_inner 1e-6,
   max_iter 20000; MIXED -> tol 1e-10, tol_T 1e-7, tol_inner 1e-1, max_iter 3000
   (a system that needs more, or whose FP32 recurrence stalls, is solved again
   in FP64 from zero);
   both: tol_adjoint 0 (= tol), max_outer 64, graphs on (16 iterations per
   replay), timing off. */
void rsn_default_opts(int precision, rsn_solver_opts* opts);

/* Create a context on CUDA device `device`, queuing work on `cuda_stream`
   (a cudaStream_t; NULL = the legacy default stream).  *out receives the
   context.  Errors: RSN_EINVAL (out NULL), RSN_ECUDA (no such device). */
rsn_status rsn_create(rsn_ctx** out, int device, void* cuda_stream);

/* Free every device and host resource of the context (NULL is a no-op). */
rsn_status rsn_destroy(rsn_ctx* ctx);

/* Grid and FD order (Sec. II.C: high-order FD Laplacian).  fd_half_order R in
   1..6 selects the order-2R central stencil (R = 1: 7-point, R = 4: 25-point,
   R = 6: 37-point).  Invalidates every other setter's data.
   Errors: RSN_EINVAL (sizes < 1, nx*ny > 4096, R out of range, h <= 0). */
rsn_status rsn_set_grid(rsn_ctx* ctx, int nx, int ny, int nz, double h, int fd_half_order);

/* Local potential V_loc (hartree), N = nx*ny*nz doubles, host memory.
   Errors: RSN_ESTATE (no grid), RSN_EINVAL (NULL). */
rsn_status rsn_set_potential(rsn_ctx* ctx, const double* v_loc);

/* Kleinman-Bylander projectors in compressed rows (Sec. II.C, nonlocal
   pseudopotential with a cutoff radius):  H_nl = sum_p e_kb[p] v_p v_p^T,
   v_p[idx[k]] = val[k] for k in offsets[p] .. offsets[p+1]-1.
   The values carry the quadrature weight (val = beta * sqrt(h^3)).  Consecutive
   projectors with identical index lists are treated as one atom (one gather).
   n_proj = 0 removes all projectors.  Host arrays.
   Errors: RSN_ESTATE (no grid), RSN_EINVAL (index out of range, offsets not
   non-decreasing, n_proj > 65536). */
rsn_status rsn_set_projectors(rsn_ctx* ctx, int n_proj, const int64_t* offsets,
                              const int32_t* idx, const double* val, const double* e_kb);

/* Absorbing potentials Gamma_L, Gamma_R >= 0 (hartree), N doubles each, host
   (Sec. II.B, Eqs. Hop and ABC).  They enter A(E) as +i(Gamma_L + Gamma_R) and
   act as the lead couplings in T.  Errors: RSN_ESTATE, RSN_EINVAL (negative). */
rsn_status rsn_set_cap(rsn_ctx* ctx, const double* gamma_l, const double* gamma_r);

/* y_k = A(E_k) x_k for n_rhs vectors (the matvec of Eqs. G/Hop: FD stencil,
   V_loc, CAP and projectors).  x_dev, y_dev: device, [n_rhs][N] complex128
   (precision RSN_FP64) or complex64 (RSN_MIXED).  E: host, n_rhs doubles.
   Errors: RSN_ESTATE, RSN_EINVAL (also n_rhs > 65535: split the call),
   RSN_ECUDA.  On an error after work was queued, the caller's stream is still
   ordered after that work. */
rsn_status rsn_apply(rsn_ctx* ctx, int precision, int n_rhs, const double* E,
                     const void* x_dev, void* y_dev);

/* Allocation-free variant of rsn_apply, for callers that must not allocate
   device memory during a call (a pre-sized memory pool, a real-time loop, or a
   host framework that owns every allocation).  The paper has no counterpart:
   this is an interface of this library only.  Same arguments and result as
   rsn_apply; it calls no cudaMalloc / cudaFree / allocating library routine.
   Its per-call scratch (launch descriptor, per-vector tables, projector
   coefficients) is a fixed 8 MiB device array that every device which loads
   the library holds until the process exits; a call whose scratch would not
   fit (n_rhs * (24 + 16 * max(n_proj, 1)) bytes plus about 1 KiB), or with
   n_rhs > 65535, fails with RSN_EINVAL before anything is queued.  The operator data must already be on the device: after the last
   setter, make one allocating call (e.g. rsn_apply) first, else RSN_ESTATE.
   The first call on a device looks up the array's device address
   (cudaGetSymbolAddress), so make it before any stream capture.  All calls
   share the array: calls that overlap on the GPU race. */
rsn_status rsn_apply_noalloc(rsn_ctx* ctx, int precision, int n_rhs, const double* E,
                             const void* x_dev, void* y_dev);

/* Green's-function columns x_{e,c} = G^r(E[e]) e_{cols[c]} (Eq. G).
   x_dev: device, [n_e][n_cols][N] complex128, written in place.  iters / relres
   (host, n_e*n_cols each, may be NULL) receive the total Krylov iterations and
   the final true relative residual; a column that did not converge gets
   iters < 0.  Errors: RSN_ESTATE, RSN_EINVAL (cols out of range), RSN_ENOMEM,
   RSN_ENOCONV / RSN_ETIMEOUT / RSN_EBREAKDOWN (x_dev still holds the best iterate). */
rsn_status rsn_solve_columns(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                             const int32_t* cols, const rsn_solver_opts* opts,
                             void* x_dev, int32_t* iters, double* relres);

/* T(E) by Eq. T-realspace restricted to the given columns:
   T[e] = 4 sum_c Gamma_R[cols[c]] sum_{i: Gamma_L,i > 0} Gamma_L,i |G_{i,cols[c]}(E[e])|^2.
   With cols = every point where Gamma_R > 0 this is the full transmission.
   T: host, n_e doubles.  Sums run in FP64 in a fixed order (bit-reproducible).
   Errors: as rsn_solve_columns (T still filled from the best iterates). */
rsn_status rsn_transmission(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                            const int32_t* cols, const rsn_solver_opts* opts, double* T);

/* Shifted COCG over an energy window: columns x_{e,c} = G^r(E[e]) e_{cols[c]}
   for every energy from ONE Krylov space per column.  A(E) = E 1 - H_op, so
   A(E[e]) = A(E_s) + (E[e] - E_s) 1 (Eq. G: the energy enters only the
   diagonal) and the COCG residuals of all the shifted systems stay collinear
   with the seed's (r_e = r / pi_e); one operator application per iteration
   serves the whole window -- the linear-solve counterpart of obtaining G over
   the whole energy range from one decomposition (Sec. II.C).  The seed E_s is
   the energy nearest the middle of the window.  FP64 only (the mixed mode's
   true-residual replacements would break the collinearity): opts->precision
   must be RSN_FP64, else RSN_EINVAL.  A shift stops once its recurrence
   residual ||r|| / |pi_e| is at most tol ||b||; shifts that have not within
   max_iter seed iterations are solved again by the plain FP64 path.
   x_dev: device, [n_e][n_cols][N] complex128 (as rsn_solve_columns).
   iters (host, n_e*n_cols, may be NULL): seed iterations at which each shift
   converged (or the plain path's count; < 0 if that failed too); relres (may
   be NULL): the recurrence estimate of the relative residual.
   Memory: the shifted directions take n_e * N complex128 per column in flight.
   Errors: as rsn_solve_columns. */
rsn_status rsn_solve_columns_shifted(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                     const int32_t* cols, const rsn_solver_opts* opts,
                                     void* x_dev, int32_t* iters, double* relres);

/* T(E) over an energy window by shifted COCG (as rsn_solve_columns_shifted):
   the shifted iterates are kept only on the support of Gamma_L, which is all
   Eq. T-realspace reads, T[e] = 4 sum_c Gamma_R[cols[c]] sum_{i in L}
   Gamma_L,i |x_{e,c}(i)|^2 (FP64, fixed order).  T: host, n_e doubles; iters
   as above (may be NULL).  Errors: as rsn_transmission; RSN_EINVAL if
   Gamma_L is zero everywhere. */
rsn_status rsn_transmission_shifted(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                    const int32_t* cols, const rsn_solver_opts* opts, double* T,
                                    int32_t* iters);

/* Block COCG: the columns of one energy, in blocks of `block` (4, 8 or 16)
   columns, each block sharing ONE block Krylov space of A(E) (A = A^T by Eq.
   complex-sym, so block CG carries over with the unconjugated bilinear form;
   the right-hand sides e_j of a block see each other's search directions).
   The paper solves one Green's-function column at a time; sharing the space
   across the right-hand sides of one energy is this library's: a block of 16
   reduces its unit columns' residuals 1e4-fold in about a third of the plain
   recurrence's iterations.
   Each block runs FP64 outer steps: the true residual R = b - A X, then an
   inner block COCG in complex FP32 on A D = R (columns scaled to unit norm)
   whose residual block is kept orthonormal (R_k = Q_k xi_k, Cholesky QR, so
   columns that converge at different rates never make the block singular),
   until every column's residual fell by tol_inner (0: 1e-4); then X += D.
   A column is done when ||b - A x|| <= tol ||b|| and, if opts->tol_T > 0,
   the change of its T partial t = sum_{i in L} Gamma_L,i |x(i)|^2 made by the
   last outer step, times ten times that step's residual reduction, is at most
   tol_T t; a block is done when all its columns are.  A block whose inner
   solve breaks down or runs long -- the first past min(max_iter, 1000)
   iterations, a restart past twice the first one's count: its FP32 block
   recurrence lost its orthogonality --, that stalls for three outer steps or
   reaches max_outer keeps its last FP64 iterate and hands its columns to the
   plain slot-pool solver of rsn_solve_columns (warm-started there, with that
   solver's FP64 re-solve of stalled systems), so every column meets the same
   targets.  opts->precision must be RSN_MIXED; deadline_ms as
   rsn_solve_columns.  cols must be distinct; a short last block of an energy
   is padded with other grid points whose solutions are dropped.
   x_dev: device, [n_e][n_cols][N] complex128 (as rsn_solve_columns);
   t_cols (host, n_e*n_cols, may be NULL): each column's T partial t;
   iters (host, may be NULL): operator applications of the column's block
   (inner iterations plus FP64 residuals) plus the plain solver's iterations
   of a handed-back column; < 0 if the column did not converge;
   relres (host, may be NULL): final ||b - A x|| / ||b||.
   Errors: RSN_EINVAL (block not 4/8/16, precision, tol_inner outside (0, 1),
   repeated columns, a grid of fewer than 2 block points, as rsn_solve_columns);
   RSN_ENOCONV (a handed-back column failed in the plain solver too; outputs
   still written); RSN_ETIMEOUT; RSN_ENOMEM / RSN_ECUDA.
   rsn_last_stats: krylov_iters = block operator applications summed over the
   columns plus the plain solver's iterations, fp64_fallbacks = the columns
   handed to the plain solver. */
rsn_status rsn_solve_columns_block(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                   const int32_t* cols, int block, double tol_inner,
                                   const rsn_solver_opts* opts, void* x_dev, double* t_cols,
                                   int32_t* iters, double* relres);

/* T(E) by Eq. T-realspace from block COCG columns (as rsn_solve_columns_block,
   without storing the columns): T[e] = 4 sum_c Gamma_R[cols[c]] t_{e,c}, FP64
   in a fixed order.  T: host, n_e doubles; t_cols, iters: as above (may be
   NULL).  Errors: as rsn_solve_columns_block. */
rsn_status rsn_transmission_block(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                  const int32_t* cols, int block, double tol_inner,
                                  const rsn_solver_opts* opts, double* T, double* t_cols,
                                  int32_t* iters);

/* T(E) as rsn_transmission, keeping the forward columns: x_dev (device,
   [n_e][n_cols][N] complex128, caller-owned) receives x_{e,c} = G(E[e]) e_{cols[c]}
   so that a later rsn_transmission_vjp_reuse needs only the adjoint solves.
   T: host, n_e doubles.  Errors: as rsn_transmission. */
rsn_status rsn_transmission_keep(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                 const int32_t* cols, const rsn_solver_opts* opts, void* x_dev,
                                 double* T);

/* Vector-Jacobian product of T with respect to V_loc from given forward columns
   (as written by rsn_transmission_keep with the same E, cols and potential):
   dV[r] = sum_e T_bar[e] 8 sum_c Gamma_R,c Re(lambda_{e,c}(r) x_{e,c}(r)) with one
   adjoint solve lambda = G (Gamma_L o conj(x)) per column (G^T = G, Eq.
   complex-sym) -- the forward columns are reused, not solved again.
   x_dev: device [n_e][n_cols][N] complex128, read only.  dV: host or device
   (dV_is_device) N doubles, overwritten.  Errors: as rsn_transmission_vjp. */
rsn_status rsn_transmission_vjp_reuse(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                      const int32_t* cols, const rsn_solver_opts* opts,
                                      const void* x_dev, const double* T_bar, double* dV,
                                      int dV_is_device);

/* T(E) of several junctions at once (many junctions, energies and column sets
   of uneven sizes; each junction is Eq. T-realspace on its own context):
   ctxs[k] holds junction k (distinct contexts, all set up); it gets n_e[k]
   energies E[k] and n_cols[k] columns cols[k], and T[k] (host, n_e[k] doubles)
   receives its T as rsn_transmission would.  When every context is on the same
   device with the same FD order and opts->rhs_block is 0, all (junction,
   energy, column) systems wait in ONE queue of one slot pool owned by ctxs[0]
   (its stream, slots and captured graphs): each slot works on its system's
   junction with that junction's tiling, and every launch of the solver serves
   all junctions; junctions whose planes need different operator kernels run
   them side by side.  The pool runs all junctions or none: if any junction's
   arguments are refused, every junction reports RSN_EINVAL.  Otherwise each
   context solves on its own stream from its own host thread (its slot pool
   capped by its share of the free device memory).  opts may be NULL (RSN_MIXED
   defaults).  status (n_ctx entries, may be NULL) receives each junction's
   result; the call returns RSN_OK if all succeeded, else the first failing
   junction's status (its message is in rsn_last_error(ctxs[k])).
   Errors: RSN_EINVAL (NULL arrays, a repeated context); as rsn_transmission per
   junction.  The paper treats one junction at a time; batching is this
   library's. */
rsn_status rsn_batch_transmission(int n_ctx, rsn_ctx* const* ctxs, const int* n_e, const double* const* E,
                                  const int* n_cols, const int32_t* const* cols, const rsn_solver_opts* opts,
                                  double* const* T, rsn_status* status);

/* Vector-Jacobian product of T with respect to V_loc:
   dV[r] = sum_e T_bar[e] dT(E[e])/dV_loc(r)
         = sum_e T_bar[e] 8 sum_c Gamma_R,c Re(lambda_{e,c}(r) x_{e,c}(r)),
   lambda = G (Gamma_L o conj(x)) -- one adjoint solve per column with the same
   operator, since G^T = G (Eq. complex-sym).  T_bar: host, n_e doubles.
   dV: host or device (dV_is_device) N doubles, overwritten.  T: host n_e
   doubles or NULL (receives T(E) of the forward pass).  Errors: as above. */
rsn_status rsn_transmission_vjp(rsn_ctx* ctx, int n_e, const double* E, int n_cols,
                                const int32_t* cols, const rsn_solver_opts* opts,
                                const double* T_bar, double* dV, int dV_is_device,
                                double* T);

/* Landauer current (Sec. II.A, Eq. Landauer):
     I(V_k) = (2e/h) int T(E) [f(E - mu_L) - f(E - mu_R)] dE,  mu_{L,R} = E_F +- V_k / 2,
   f the Fermi-Dirac occupation at temperature kT (hartree; kT = 0: a step with
   f(0) = 1/2).  Atomic units: e = hbar = 1, so 2e/h = 1/pi, energies and the
   bias eV in hartree, I in e E_h / hbar (6.62 mA); the factor 2 is the spin.
   The integral is the trapezoidal rule on the grid E (host, n_e strictly
   ascending doubles) with T (host, n_e doubles, e.g. from
   rsn_transmission_shifted); T is taken as zero outside the grid.  One kernel
   on the context's stream, FP64, fixed-order sums.  I: host, n_v doubles.
   Errors: RSN_EINVAL (NULL, unsorted or non-finite input, kT < 0). */
rsn_status rsn_landauer_current(rsn_ctx* ctx, int n_e, const double* E, const double* T, int n_v,
                                const double* V, double E_F, double kT, double* I);

/* Counters of the last solve on this context: total Krylov iterations over all
   systems, true-residual replacements (reliable updates), device kernel
   launches queued, elapsed GPU milliseconds of the solve phase, and the number
   of systems that RSN_MIXED solved again in FP64 because the FP32 recurrence
   stalled (a near-singular A(E): the FP32 operator error times the condition
   number approaches 1) or because the mixed pass stopped early when most of
   its finished systems had stalled.  Any pointer may be NULL. */
rsn_status rsn_last_stats(const rsn_ctx* ctx, int64_t* krylov_iters, int64_t* sweeps,
                          int64_t* launches, double* gpu_ms, int64_t* fp64_fallbacks);

/* Live per-kernel timing of the last solve call made with opts.timing = 1.
   kind 0: the fused COCG operator kernel (p = r + beta p, q = A p, p^T q);
   kind 1: the COCG update kernel (projector term of q on the support points,
   r -= alpha q, d += alpha p, r^T r).
   launches: launches timed; ms: summed CUDA-event durations on the library's
   stream; bytes: algorithmic HBM bytes of those launches (vectors read and
   written once per active system: 4 vectors for kind 0, 6 for kind 1).
   Any output pointer may be NULL.  Errors: RSN_EINVAL (kind). */
rsn_status rsn_kernel_stats(const rsn_ctx* ctx, int kind, int64_t* launches, double* ms,
                            double* bytes);

/* Micro-benchmark of one kernel of the COCG iteration on `nslots` systems of
   the current junction, all active with a synthetic finite state (results are
   meaningless, timings are not).  kind 0: fused operator kernel (p update,
   stencil, V/CAP, projectors, p^T A p); kind 1: COCG update kernel; kind 2:
   FP64 true-residual kernel.  Runs 2 untimed then `reps` timed launches on the
   context's stream (CUDA events).  ms_per_launch: mean duration;
   bytes_per_launch: algorithmic HBM bytes of one launch (each vector read or
   written once per point).  Errors: RSN_ESTATE, RSN_EINVAL, RSN_ENOMEM. */
rsn_status rsn_bench_kernel(rsn_ctx* ctx, int precision, int kind, int nslots, int reps,
                            double* ms_per_launch, double* bytes_per_launch);

/* Autotuner: times the fused operator kernel (rsn_bench_kernel kind 0) for a
   set of tilings of this grid -- the FP32 plane kernel, the point-pair kernel
   and the whole-plane bulk-copy kernel with several z-chunk lengths, and the
   register-prefetch kernel over rows per tile, points per thread and z-chunks
   -- and keeps on the context the one with the least launch time with all
   nslots systems active plus with a quarter of them active (the tail of a
   solve, where long z chunks leave SMs idle).  Outputs (any may be NULL): the
   chosen TY, Lz, ppt (0 = automatic), tma (3: the plane kernel, 2: the
   point-pair kernel, 1: the whole-plane bulk-copy kernel, 0: the register
   kernel) and its algorithmic GB/s.  Errors: as rsn_bench_kernel; RSN_ECUDA
   if no candidate ran. */
rsn_status rsn_autotune(rsn_ctx* ctx, int precision, int nslots, int* TY, int* Lz, int* ppt,
                        int* tma, double* best_gbs);

/* Override the operator kernel's tile (0 = automatic).  Automatic, for FP32
   operators: with nx even and planes of at most 1280 points, the point-pair
   kernel (two x-neighbours per thread, whole planes streamed by bulk copies
   through a ring of shared-memory stages, a register ring of 2R+1 planes,
   two CTAs per SM up to 576 points); else, for planes of an even number of at
   most 576 points, the plane kernel (the same with one point per thread);
   everything else, and FP64, the register-prefetch kernel.  Lz sets the
   planes per CTA of any of them.  TY rows of the x-y plane per CTA and ppt
   owned points per thread (1..4) select the register-prefetch kernel; ppt = -1
   the whole-plane bulk-copy kernel with a shifted register queue (FP32, planes
   of at most 1024 points with 16-byte aligned sizes); ppt = -2 the point-pair
   kernel; ppt = -3 the plane kernel.  Cases a choice does not support keep the
   next kernel in this order.  The FP64 true-residual kernel takes TY and ppt but
   always works on two planes per CTA.  Used by the autotuner and by tests that
   force ragged tiles; it does not change results beyond rounding order.
   Errors: RSN_EINVAL. */
rsn_status rsn_set_tiling(rsn_ctx* ctx, int TY, int Lz, int ppt);

/* Human-readable description of the context's last error ("" if none).
   ctx may be NULL (reports errors from rsn_create). */
const char* rsn_last_error(const rsn_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RSNEGF_H */
