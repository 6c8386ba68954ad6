// Internal structures shared by the library's translation units.
//
// Data layout in device memory (per junction, N = nx*ny*nz points, x fastest):
//   dg64/dg32   (N)  complex diagonal without E: (-V_loc + 3 c_0/(2h^2), Gamma_L+Gamma_R)
//   gl          (N)  Gamma_L (FP64), used by T and the adjoint right-hand side
//   inv_*            per-point list of (projector, value) for the matvec epilogue
//   grp_*            per-atom support lists for the projections c_p = v_p . x
// Krylov vectors of one batch are stored column-contiguous: slot s owns
// elements [voff[s], voff[s] + N) of every vector array.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rsn {

constexpr int kMaxR = 6;        // up to the order-12 stencil
constexpr int kMaxPlane = 4096; // nx*ny limit (smem plane tiles)
constexpr int kMaxGroupNp = 16; // projectors per atom (s,p,d = 9)
constexpr int kVecThreads = 256;
constexpr int kVecPerThread = 8;   // points per thread in the streaming kernels
constexpr int kVecPts = kVecThreads * kVecPerThread;

struct JuncDev {
  int nx, ny, nz, plane;
  long long N;
  // stencil tiling of the operator kernel for this junction
  int TY, Lz, ytiles, ztiles, nA;  // nA = ytiles*ztiles CTAs per slot (this launch's tiling)
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
  const int* inv_ptr;
  const int* inv_proj;
  const double* inv_val64;
  const float* inv_val32;
  const int* grp_ptr;
  const int* grp_p0;
  const int* grp_np;
  const long long* grp_voff;
  const int* grp_idx;
  const double* grp_val64;
  const float* grp_val32;
  const double* ekb;
};

// Per-slot state of a batch of systems A(E_s) x_s = b_s.
struct BatchDev {
  int nslots;
  int PA, PB;  // partial-sum strides per slot (>= nA, nB of every junction)
  const int* junc;
  const double* E;
  const int* col;          // >= 0: b = e_col ; -1: adjoint b = Gamma_L o conj(xf)
  const long long* voff;
  double2* x64;
  const double2* xf;
  void* r;
  void* p0;
  void* p1;
  void* q;
  void* d;
  int* iters;       // Krylov iterations since the last restart
  int* done;        // inner solve finished (or slot idle)
  int* outer_done;  // slot finished for good
  int* total_iters;
  int* n_outer;
  int* status;      // 0 ok, 1 no-conv, 2 breakdown seen
  int* breakdowns;
  double* bnorm2;
  double* tol2;
  double* relres;
  double2* rho0_part;  // [nslots][PA] rho_0 from the true-residual kernel
  double* nrm0_part;   // [nslots][PA]
  double2* rho_part;   // [2][nslots][PB]
  double* nrm_part;    // [nslots][PB]
  double2* mu_part;    // [nslots][PA]
  void* c_r;           // [nslots][n_proj] projections of r (inner precision)
  void* c_p;           // [2][nslots][n_proj] projections of p
  double2* c_x;        // [nslots][n_proj] projections of x64 + d (FP64)
  int* n_active;       // [2]: inner active count, outer active count
};

enum OpMode { OP_COCG = 0, OP_RESID = 1, OP_APPLY = 2 };

struct OpLaunch {
  int threads;  // CTA size
  int ppt;      // owned points per thread
  size_t smem;  // dynamic shared memory bytes
};

// ---- launchers (defined in the .cu files) --------------------------------
// operator kernels (ops_r<R>.cu)
cudaError_t launch_op(int mode, bool fp32, int R, int ppt, dim3 grid, int threads, size_t smem,
                      cudaStream_t st, const JuncDev* jt, const BatchDev& b, const void* x_in,
                      void* y_out, const void* c_in);
size_t op_smem_bytes(bool fp32, int mode, int R, int TY, int nx, int n_proj);

// streaming / reduction kernels (vec_kernels.cu)
cudaError_t launch_cocg_update(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt,
                               const BatchDev& b);
cudaError_t launch_project(int mode, bool fp32, int nslots, int n_groups, cudaStream_t st,
                           const JuncDev* jt, const BatchDev& b, const void* x_in, void* c_out);
cudaError_t launch_inner_book(int nslots, int max_iter, cudaStream_t st, const JuncDev* jt,
                              const BatchDev& b);
cudaError_t launch_outer_book(int nslots, double tol, double tol_inner, int max_outer,
                              cudaStream_t st, const JuncDev* jt, const BatchDev& b);
cudaError_t launch_x_update(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt,
                            const BatchDev& b);
cudaError_t launch_bnorm_adjoint(int nslots, cudaStream_t st, const JuncDev* jt, const BatchDev& b);
cudaError_t launch_t_partial(int nslots, cudaStream_t st, const JuncDev* jt, const BatchDev& b,
                             const int* out_index, double* t_out);
cudaError_t launch_t_final(int n_e, int n_cols, cudaStream_t st, const double* t_all,
                           const double* gr_cols, double* T_out);
cudaError_t launch_grad_accum(int nslots, long long N, cudaStream_t st, const BatchDev& b,
                              const double* wt, double* g);

}  // namespace rsn
