// Internal structures shared by the library's translation units.
//
// Data layout in device memory (per junction, N = nx*ny*nz points, x fastest):
//   dg64        (N)  complex diagonal without E: (-V_loc + 3 c_0/(2h^2), Gamma_L+Gamma_R)
//   dg32        (N)  (-V_loc, Gamma_L+Gamma_R) for the FP32 difference-form stencil
//   gl          (N)  Gamma_L (FP64), used by T and the adjoint right-hand side
//   inv_*            per-point list of (projector, value) for the matvec epilogue
//   grp_*            per-atom support lists for the projections c_p = v_p . x
// Krylov vectors (r, p0, p1, q, d) are stored per slot: slot s owns elements
// [voff[s], voff[s] + N) of each array.  The FP64 iterate of the system held by
// slot s lives at x64[xo[s] ...], the forward solution an adjoint system reads at
// xf[xfo[s] ...].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rsn {

constexpr int kMaxR = 6;        // up to the order-12 stencil
constexpr int kMaxPlane = 4096; // nx*ny limit (smem plane tiles)
constexpr int kMaxGroupNp = 16; // projectors per atom (s,p,d = 9)
// zero entries after the n_proj projector coefficients in shared memory, read
// by the zero-padded tail of an atom's last value quad
constexpr int kCePad = 16;
constexpr int kMaxGraphIters = 256;
constexpr int kMaxApplyRhs = 65535;  // vectors per operator-application call (grid y dimension)
constexpr int kMaxGoalChecks = 24;   // T checks of a goal phase before it ends
constexpr int kSchedThreads = 1024;
// CTA rows of the kernels that work only on NEW / CHECK slots (zero, true
// residual and its projections, x update): each row takes list entries
// row, row + kListRows, ...; a handful of slots need them per iteration
constexpr int kListRows = 32;
// systems past the first unstarted one that the scheduler examines for a
// ready system (its dependency finished) when slots are free
constexpr int kReadyWindow = 4096;
constexpr int kVecThreads = 256;
constexpr int kVecPerThread = 16;  // points per thread in the streaming kernels
constexpr int kVecPts = kVecThreads * kVecPerThread;

struct JuncDev {
  int nx, ny, nz, plane;
  long long N;
  // stencil tiling of the operator kernel for this junction
  int TY, Lz, ytiles, ztiles, nA;  // nA = ytiles*ztiles CTAs per slot (this launch's tiling)
  int kind;                        // operator kernel of this junction's slots: kOpReg, kOpTma, kOpPair, kOpPlane
  int nR;                          // CTAs per slot of the true-residual kernel (rho_0, ||r_0||^2 partials)
  int nB;                          // streaming-kernel CTAs per slot
  double w64[kMaxR + 1];           // w[m] = c_m / (2 h^2), m = 1..R (w[0] unused)
  float w32[kMaxR + 1];
  const double2* dg64;
  const float2* dg32;
  const double* gl;
  int nL;
  const int* L_idx;
  const double* L_gam;
  // projectors
  int n_proj, n_groups;
  // per grid point i, entries inv_ptr[i] .. inv_ptr[i+1]-1, one per atom whose
  // support holds i: the atom's first projector inv_p0[e] and the values of
  // its projectors at i in inv_nq quads (zero-padded), FP64 as 2 double2 per quad
  const int* inv_ptr;
  int inv_nq;
  const int* inv_p0;
  const double2* inv_q64;
  const float4* inv_q32;
  const int* sup_pts;  // the grid points with at least one entry, ascending
  int n_sup, nS;       // their number; CTAs per slot of the projector-term kernel
  const int* grp_ptr;
  const int* grp_p0;
  const int* grp_np;
  const long long* grp_voff;
  const int* grp_idx;
  const double* grp_val64;
  const float* grp_val32;
  const double* ekb;
};

// Life cycle of a slot of the streaming solver.
enum SlotState {
  SL_FREE = 0,    // no system; gets the next one from the queue
  SL_NEW = 1,     // system assigned: zero x and d, then true residual r = b
  SL_CHECK = 2,   // recurrence reached its target: FP64 true residual + reliable update
  SL_ACTIVE = 3,  // COCG iterations in the inner precision
  SL_DRAIN = 4,   // finished this iteration: outputs are emitted, then FREE
  SL_CHECKT = 5   // goal phase: the recurrence reached its next target; x += sigma d and the
                  // T partial of x are taken without touching the recurrence (no true residual)
};

// Batch state.  Lives in device memory; kernels receive a pointer to it so
// captured CUDA graphs stay valid when a call changes the buffers it points to.
struct BatchDev {
  int nslots;
  int PA, PB;  // partial-sum strides per slot (>= nA / nR and nB of every junction)
  // per slot
  int* state;
  int* sys;
  int* junc;
  double* E;
  int* col;             // >= 0: b = e_col ; -1: adjoint b = Gamma_L o conj(xf)
  long long* voff;      // inner vectors
  long long* xo;        // FP64 iterate
  long long* xfo;       // forward solution (adjoint right-hand side)
  int* iters;           // COCG iterations since the last restart (p = r at iters == 0)
  int* total_iters;
  int* cyc_iters;       // COCG iterations since the last true residual
  int* n_upd;           // reliable updates so far
  int* restart;         // breakdown seen: restart with p = r at the next update
  int* stall;           // consecutive true residuals that did not improve 4x
  int* warm;            // the system starts from the iterate already in x64
  double2* rho_cur;     // rho_k = r^T r of the current iteration (set by book / sched)
  double2* beta_cur;    // beta_k = rho_k / rho_{k-1} for the direction update of iteration k
  double* bnorm2;
  double* sigma;        // ||b||: the inner-precision vectors hold r / sigma and d / sigma
  double* rlast2;       // true ||r||^2 at the previous replacement (progress check)
  double* rrec2;        // recurrence ||r / sigma||^2 when the cycle ended (drift check)
  double* tol2;         // recurrence target ||r||^2 of the current cycle
  // vectors
  double2* x64;
  const double2* xf;
  void* r;
  void* p0;
  void* p1;
  void* q;
  void* d;
  // reduction partials
  double2* rho0_part;   // [S][PA] true-residual kernel: r^T r
  double* nrm0_part;    // [S][PA] true-residual kernel: ||r||^2
  double* t0_part;      // [S][PA] true-residual kernel: sum Gamma_L |x|^2 of the iterate (forward systems)
  double* tlast;        // [S] that sum at the previous true residual (-1: none yet)
  int* gcnt;            // [S] T checks since the residual met tol (goal phase)
  int* gphase;          // [S] 1: goal phase (the residual met tol, the T partial is converging)
  double* tgoal;        // [S] T partial of x at a goal-phase check
  double* rgoal;        // [S] relative true residual when the goal phase began
  double2* rho_part;    // [S][PB] COCG update kernel: r^T r
  double* nrm_part;     // [S][PB]
  double2* mu_part;     // [S][PA] operator kernel: p^T A p
  int pstride;          // per-slot stride of the projection arrays (the largest n_proj of the junctions)
  void* c_r;            // [S][n_proj] projections of r (inner precision)
  void* c_p;            // [2][S][n_proj] projections of p
  double2* c_x;         // [S][n_proj] projections of x64 + d (FP64)
  // systems queue and outputs
  int nsys;
  const int* sys_junc;
  const double* sys_E;
  const int* sys_col;
  const long long* sys_xo;   // x64 offset of each system (-1: slot storage)
  const long long* sys_xfo;
  const int* sys_dep;        // system that must finish first (adjoint after forward), -1 none
  const double* sys_bn2;     // known ||b||^2 of a warm-started system (> 0: warm start), may be null
  int* sys_started;          // 1 once a system has been given a slot
  int* out_iters;
  double* out_relres;
  int* out_status;           // -1 pending, 0 converged, 1 not converged, 2 breakdown,
                             // 3 stalled (precision-limited: re-solve in FP64)
  double* out_t;             // T partial sum_{i in L} Gamma_L |x(i)|^2 per system (may be null)
  int* sched;                // [0] next system, [1] busy slots, [3 + it] busy after iteration it of a
                             // replay, [3 + kMaxGraphIters + it] systems that did a COCG iteration
                             // (zeroed at the start of each replay)
  unsigned long long* counters;  // [0] COCG iterations, [1] reliable updates, [2] finished, [3] not converged
  int* lst;                  // NEW / CHECK slots of the current iteration, in slot order
  int* lst_n;                // their number
  int* inlist;               // [S] 1: the slot is in this iteration's list
  int* fslot;                // FREE slots in slot order (scheduler scratch)
  void* c_e;                 // e_kb[p] c_p[p] of the current direction per slot (inner precision),
  int ce_stride;             // n_proj + kCePad entries per slot, the last kCePad always zero
  // shifted systems: one seed Krylov space per column serves every energy of a
  // window, A(E_e) = A(E_seed) + sigma_e 1 (Eq. G); n_shift = 0 for plain solves
  int n_shift;
  const double* shift_sig;   // sigma_e = E_e - E_seed, e < n_shift
  int nT;                    // tracked points of the shifted iterates
  const int* T_idx;          // their grid indices (the Gamma_L support, or every point)
  double2* xs;               // shifted iterates x_e on the tracked points
  long long xs_sstride;      // xs offset of slot / system k: k * xs_sstride + e * xs_estride
  long long xs_estride;
  int xs_by_sys;             // 1: xs is indexed by system (caller's output), 0: by slot
  double2* ps;               // shifted directions p_e: [slot][n_shift][nT]
  double2* spi;              // pi_{e,k} ring: [3][slot][n_shift], iteration k in ring k % 3
  int* sconv_it;             // [slot][n_shift] iteration at which shift e converged (INT_MAX: not yet)
  double2* salpha;           // [2][slot] alpha_k of the seed recurrence, ring k % 2
  double2* sbeta;            // [2][slot] beta_k, ring k % 2
  double* rn2;               // [slot] ||r_{k+1}||^2 of the seed (bookkeeping kernel)
  double* out_ts;            // [n_shift][system] T partial sum_{i in L} Gamma_L |x_e(i)|^2
  int* out_sit;              // [n_shift][system] seed iterations at convergence (-1: not converged)
  double* out_srel;          // [n_shift][system] recurrence estimate ||r_k|| / |pi_{e,k}| / ||b||
  // options
  double tol, delta;
  double tol_adj;  // tolerance of systems with a computed right-hand side (col < 0)
  double tol_T;    // forward systems also finish only once sum Gamma_L |x|^2 changed by at most
                   // tol_T of itself between two true residuals (0: residual criterion alone)
  int max_iter, max_upd;
  int cycle_cap;  // a cycle longer than this ends with a true residual even if its target was not met
  int stall_cap;  // true residuals in a row without a 4x gain before a system is handed back (0 = never)
  int handback;   // 1: systems whose predicted iteration count exceeds max_iter are handed back early
};

// Block COCG: the B columns of one energy share one block Krylov space
// (A(E) = A(E)^T, so the COCG recurrence carries over to blocks with the
// unconjugated bilinear form).  The residual block is kept orthonormal,
// R_k = Q_k xi_k with Q_k = W_k tau_k^{-1} (Cholesky QR of W_k), so columns
// that converge at different rates do not make the b x b systems singular.
// The block recurrence runs in complex FP32; the b x b algebra in FP64; an FP64
// true residual restarts it (defect correction) until every column meets its
// residual and T-partial targets.
constexpr int kBlkThreads = 256;  // vector kernels and the Gram kernel
constexpr int kBlkTile = 64;      // points per shared-memory tile of the Gram kernel
constexpr int kBlkMax = 16;       // largest block
constexpr int kBlkInnerCap = 1000; // iterations of one inner solve before it is abandoned

struct BlkDev {
  int B;                  // columns per block (4, 8 or 16)
  long long N;
  int nchunk;             // Gram partial sums per block
  long long chunk_pts;    // points per Gram chunk (a multiple of kBlkTile)
  int nchunkR;            // residual partial sums per vector
  long long chunkR_pts;
  const int* icap;        // [nb] inner iterations before an inner solve of the block ends unconverged
  double tol_in;          // inner solve: each column's residual reduced by this factor
  const int* blist;       // blocks of this launch (grid.y), host-compacted
  const int* col;         // [nb*B] right-hand side e_col of each member
  const double* gl;       // Gamma_L
  // b x b state per block, row-major [row * B + col]
  double2* xi;            // R_k = Q_k xi_k
  double2* QQ;            // Q_k^T Q_k
  double* xi0n;           // [nb][B] column norms of xi_0
  double2* part;          // [nb][nchunk][2][B*B] Gram partials
  float2* alpha;          // alpha_k = (P^T A P)^{-1} Q^T Q
  float2* axi;            // alpha_k xi_k
  float2* tinv;           // tau_k^{-1} (upper triangular)
  double2* tinv64;        // tau_0^{-1} of a restart (FP64)
  float2* beta;           // beta_k = (Q_k^T Q_k)^{-1} tau_{k+1}^T Q_{k+1}^T Q_{k+1}
  int* flag;              // [nb] 0 iterating, 1 converged, 2 breakdown, 3 iteration cap
  int* its;               // [nb] iterations of the current inner solve
  // vectors: member a of block k at ((k * B + a) * N)
  float2* W;
  float2* P;
  float2* AP;
  float2* D;              // inner solution (correction of the normalised residual block)
  double2* X;             // FP64 iterate
  double2* R;             // FP64 residual b - A X (the FP64 operator writes A X here first),
                          // normalised per member at a restart
  double* rpart;          // [nb*B][nchunkR][2] partials of ||r||^2 and sum Gamma_L |x|^2
  double* rn;             // [nb*B] ||r|| of the current outer step
  double* tt;             // [nb*B] sum_{i in L} Gamma_L |x(i)|^2
};

cudaError_t launch_blk_comb_p(int B, int nb, cudaStream_t st, const BlkDev* d, long long N);
cudaError_t launch_blk_comb_w(int B, int nb, cudaStream_t st, const BlkDev* d, long long N);
cudaError_t launch_blk_gram(int B, int mode, int nb, int nchunk, cudaStream_t st, const BlkDev* d);
cudaError_t launch_blk_small(int B, int phase, int nb, cudaStream_t st, const BlkDev* d);
cudaError_t launch_blk_gram64(int B, int nb, int nchunk, cudaStream_t st, const BlkDev* d);
cudaError_t launch_blk_q0(int B, int nb, cudaStream_t st, const BlkDev* d, long long N);
// outer step kernels over the members of the listed blocks
cudaError_t launch_blk_resid(int B, int nb, int nchunkR, bool have_ax, cudaStream_t st, const BlkDev* d);
cudaError_t launch_blk_norm(int B, int nb, int nchunkR, cudaStream_t st, const BlkDev* d);
cudaError_t launch_blk_scale(int B, int nb, cudaStream_t st, const BlkDev* d, long long N);
cudaError_t launch_blk_xupd(int B, int nb, cudaStream_t st, const BlkDev* d, long long N);

enum OpMode { OP_COCG = 0, OP_RESID = 1, OP_APPLY = 2 };
// operator kernels; a slot pool over several junctions launches each kind its
// junctions use, and every kernel skips the slots of junctions of another kind
enum OpKind { kOpReg = 0, kOpTma = 1, kOpPair = 2, kOpPlane = 3 };

// ---- launchers (defined in the .cu files) --------------------------------
cudaError_t launch_op(int mode, bool fp32, int R, int ppt, dim3 grid, int threads, size_t smem,
                      cudaStream_t st, const JuncDev* jt, const BatchDev* b, const void* x_in,
                      void* y_out, const void* c_in);
size_t op_smem_bytes(bool fp32, int mode, int R, int TY, int nx, int n_proj);
// plane-streaming (TMA) operator kernel for whole-plane tiles (OP_COCG / OP_APPLY)
cudaError_t launch_op_tma(int mode, bool fp32, int R, dim3 grid, int threads, size_t smem, cudaStream_t st,
                          const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in);
size_t op_tma_smem_bytes(bool fp32, int mode, int R, int nx, int ny, int n_proj);
// FP32 point-pair operator kernel with plane streaming (OP_COCG / OP_APPLY):
// whole planes, nx even, 16-byte aligned vectors; big: the one-CTA-per-SM
// variant for planes of more than 2 * kPairThreads points
constexpr int kPairThreads = 288;     // threads per CTA of the two-CTAs-per-SM variant
constexpr int kPairThreadsBig = 640;  // one CTA per SM (planes of up to 1280 points)
constexpr int kPairStages = 4;        // input planes in flight per CTA
constexpr int kPlaneThreads = 576;    // one-point-per-thread plane kernel: threads per CTA (two per SM)
constexpr int kPairXO = 8;            // zero columns left of x = 0 in the exchange tile (>= R, even)
cudaError_t launch_op_pair(int mode, int R, bool big, dim3 grid, int threads, size_t smem, cudaStream_t st,
                           const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in);
size_t op_pair_smem_bytes(int mode, int R, int nx, int ny, int n_proj);
// FP32 one-point-per-thread kernel with plane streaming: whole planes of an
// even number of at most kPlaneThreads points; same shared-memory layout
cudaError_t launch_op_plane(int mode, int R, dim3 grid, int threads, size_t smem, cudaStream_t st, const JuncDev* jt,
                            const BatchDev* b, const void* x_in, void* y_out, const void* c_in);

cudaError_t launch_zero(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt, const BatchDev* b);
// the COCG update with the projector term of q on the support points; ce_stride:
// per-slot entries of e_kb c_p (BatchDev::ce_stride), staged in shared memory
cudaError_t launch_cocg_update(bool fp32, int nslots, int nB, int ce_stride, cudaStream_t st, const JuncDev* jt,
                               const BatchDev* b);
cudaError_t launch_project(int mode, bool fp32, int nslots, int n_groups, int max_np, cudaStream_t st,
                           const JuncDev* jt, const BatchDev* b, const void* x_in, void* c_out,
                           bool one_slot_per_cta = false);
cudaError_t launch_book(int nslots, int slot_it, cudaStream_t st, const JuncDev* jt, const BatchDev* b);
constexpr int kBookWarps = 8;  // slots per CTA of the bookkeeping kernel (one warp each)
cudaError_t launch_sched(int nslots, int slot_it, cudaStream_t st, const JuncDev* jt, const BatchDev* b);
cudaError_t launch_x_update(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt,
                            const BatchDev* b);
cudaError_t launch_emit(int nslots, cudaStream_t st, const JuncDev* jt, const BatchDev* b);
cudaError_t launch_list(cudaStream_t st, const BatchDev* b);
cudaError_t launch_landauer(int n_e, const double* E, const double* T, int n_v, const double* V, double E_F,
                            double kT, double* I, cudaStream_t st);
cudaError_t launch_tgoal(cudaStream_t st, const JuncDev* jt, const BatchDev* b);
cudaError_t launch_t_final(int n_e, int n_cols, cudaStream_t st, const double* t_all,
                           const double* gr_cols, double* T_out);
// shifted systems: initialisation of NEW slots, the per-iteration update of
// the shifted iterates (after the bookkeeping kernel) and their T partials
cudaError_t launch_shift_init(int nT, cudaStream_t st, const JuncDev* jt, const BatchDev* b);
cudaError_t launch_shift_update(int nslots, int nT, int n_shift, cudaStream_t st, const JuncDev* jt,
                                const BatchDev* b);
cudaError_t launch_shift_emit(int nslots, int n_shift, cudaStream_t st, const JuncDev* jt, const BatchDev* b);
cudaError_t launch_grad_sys(int nsys, long long N, cudaStream_t st, const double2* lam, const double2* x,
                            const double* wt, double* g);

}  // namespace rsn
