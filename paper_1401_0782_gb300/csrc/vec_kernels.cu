// Streaming and reduction kernels of the batched COCG solve, the T(E)
// reduction (Eq. T-realspace) and the adjoint gradient.
#include <type_traits>

#include "cplx.cuh"
#include "ops_kernel.cuh"
#include "rsn_internal.h"

namespace rsn {

// ---------------------------------------------------------------------------
// COCG update (after the operator kernel of the same iteration):
//   alpha = rho_k / mu_k,  r -= alpha q,  d += alpha p_new   (d = alpha p at k = 0)
//   partial sums of rho_{k+1} = r^T r and ||r||^2.
// Each CTA covers kVecPts consecutive points of one system.  A non-finite
// alpha leaves r and d untouched and flags the slot through a NaN norm.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cocg_update_kernel(const JuncDev* __restrict__ jt,
                                                                  const BatchDev b) {
  using C = typename cx<T>::t;
  const int s = blockIdx.y;
  if (b.done[s]) return;
  const JuncDev& J = jt[b.junc[s]];
  if ((int)blockIdx.x >= J.nB) return;
  __shared__ double red[32 * 3];
  const int k = b.iters[s];
  double2 mu = make_double2(0.0, 0.0);
  {
    const double2* mp = b.mu_part + (size_t)s * b.PA;
    for (int t = 0; t < J.nA; ++t) { mu.x += mp[t].x; mu.y += mp[t].y; }
  }
  const double2 a64 = cdiv(slot_rho(b, J, s, k), mu);
  const size_t slot_out = ((size_t)((k + 1) & 1) * b.nslots + s) * b.PB + blockIdx.x;
  if (!isfinite(a64.x) || !isfinite(a64.y)) {
    if (threadIdx.x == 0) {
      b.nrm_part[(size_t)s * b.PB + blockIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
      b.rho_part[slot_out] = make_double2(0.0, 0.0);
    }
    return;
  }
  const C alpha = from64<C>(a64);
  const long long vo = b.voff[s];
  const C* pn = reinterpret_cast<const C*>((k & 1) ? b.p0 : b.p1);
  const C* qv = reinterpret_cast<const C*>(b.q);
  C* rv = reinterpret_cast<C*>(b.r);
  C* dv = reinterpret_cast<C*>(b.d);
  const long long i0 = (long long)blockIdx.x * kVecPts;
  const long long i1 = min(i0 + (long long)kVecPts, J.N);
  T nrm = 0, rre = 0, rim = 0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
    const long long g = vo + i;
    const C p = pn[g];
    const C q = qv[g];
    C r = rv[g];
    r.x -= alpha.x * q.x - alpha.y * q.y;
    r.y -= alpha.x * q.y + alpha.y * q.x;
    C d = (k == 0) ? czero<C>() : dv[g];
    d = cfma(alpha, p, d);
    rv[g] = r;
    dv[g] = d;
    nrm = fma(r.x, r.x, fma(r.y, r.y, nrm));
    rre = fma(r.x, r.x, fma(-r.y, r.y, rre));
    rim = fma((T)2 * r.x, r.y, rim);
  }
  T v[3] = {nrm, rre, rim};
  double out[3];
  block_sum<3>(v, red, out);
  if (threadIdx.x == 0) {
    b.nrm_part[(size_t)s * b.PB + blockIdx.x] = out[0];
    b.rho_part[slot_out] = make_double2(out[1], out[2]);
  }
}

// ---------------------------------------------------------------------------
// Projections c_p = v_p . v for every projector, one CTA per (atom, system):
// the atom's support is gathered once and dotted with each of its projectors.
//   PJ_R: v = r (inner precision)           -> c_r   (skip finished inner solves)
//   PJ_X: v = x64 + d (FP64)                -> c_x   (skip finished systems)
//   PJ_IN: v = x_in (apply entry point)     -> c_out
// ---------------------------------------------------------------------------
enum { PJ_R = 0, PJ_X = 1, PJ_IN = 2 };

template <typename T, int MODE>
__global__ void __launch_bounds__(128) project_kernel(const JuncDev* __restrict__ jt, const BatchDev b,
                                                      const void* __restrict__ x_in,
                                                      void* __restrict__ c_out) {
  using CT = typename std::conditional<MODE == PJ_X, double, T>::type;
  using C = typename cx<CT>::t;
  using CO = typename cx<T>::t;
  const int g = blockIdx.x, s = blockIdx.y;
  if (MODE == PJ_R && b.done[s]) return;
  if (MODE == PJ_X && b.outer_done[s]) return;
  const JuncDev& J = jt[b.junc[s]];
  if (g >= J.n_groups) return;
  __shared__ double red[32 * 2];
  const int p0 = J.grp_p0[g], np = J.grp_np[g];
  const int k0 = J.grp_ptr[g], k1 = J.grp_ptr[g + 1], len = k1 - k0;
  const long long vb = J.grp_voff[g];
  const long long vo = b.voff[s];
  C acc[kMaxGroupNp];
#pragma unroll
  for (int p = 0; p < kMaxGroupNp; ++p) acc[p] = czero<C>();
  for (int kk = k0 + threadIdx.x; kk < k1; kk += blockDim.x) {
    const long long gi = vo + J.grp_idx[kk];
    C v;
    if constexpr (MODE == PJ_R) {
      v = reinterpret_cast<const CO*>(b.r)[gi];
    } else if constexpr (MODE == PJ_X) {
      const double2 xx = b.x64[gi];
      const double2 dd = to64(reinterpret_cast<const CO*>(b.d)[gi]);
      v = mk2(xx.x + dd.x, xx.y + dd.y);
    } else {
      v = reinterpret_cast<const CO*>(x_in)[gi];
    }
    const long long vk = vb + (kk - k0);
#pragma unroll
    for (int p = 0; p < kMaxGroupNp; ++p) {
      if (p < np) {
        const CT a = (sizeof(CT) == 8) ? (CT)J.grp_val64[vk + (long long)p * len]
                                       : (CT)J.grp_val32[vk + (long long)p * len];
        acc[p] = rfma(a, v, acc[p]);
      }
    }
  }
  C* out = reinterpret_cast<C*>(c_out) + (size_t)s * J.n_proj + p0;
  for (int p = 0; p < np; ++p) {
    CT v[2] = {acc[p].x, acc[p].y};
    double o[2];
    block_sum<2>(v, red, o);
    if (threadIdx.x == 0) out[p] = mk2((CT)o[0], (CT)o[1]);
  }
}

// ---------------------------------------------------------------------------
// Bookkeeping after each COCG iteration (one CTA): iteration counts, inner
// convergence on the recurrence residual, breakdown detection, active count.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) inner_book_kernel(const JuncDev* __restrict__ jt, const BatchDev b,
                                                          int max_iter) {
  __shared__ double red[32];
  int active = 0;
  for (int s = threadIdx.x; s < b.nslots; s += blockDim.x) {
    if (b.done[s]) continue;
    const JuncDev& J = jt[b.junc[s]];
    const int k = b.iters[s] + 1;
    b.iters[s] = k;
    b.total_iters[s] += 1;
    double nrm = 0.0;
    const double* np = b.nrm_part + (size_t)s * b.PB;
    for (int t = 0; t < J.nB; ++t) nrm += np[t];
    double2 mu = make_double2(0.0, 0.0);
    const double2* mp = b.mu_part + (size_t)s * b.PA;
    for (int t = 0; t < J.nA; ++t) { mu.x += mp[t].x; mu.y += mp[t].y; }
    const bool bad = !isfinite(nrm) || !(mu.x != 0.0 || mu.y != 0.0);
    if (bad) {
      b.done[s] = 1;
      b.breakdowns[s] += 1;
    } else if (nrm <= b.tol2[s] || k >= max_iter) {
      b.done[s] = 1;
    }
    active += b.done[s] ? 0 : 1;
  }
  double v[1] = {(double)active};
  double out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) b.n_active[0] = (int)out[0];
}

// ---------------------------------------------------------------------------
// Refinement bookkeeping after the FP64 true residual (one CTA).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) outer_book_kernel(const JuncDev* __restrict__ jt, const BatchDev b,
                                                          double tol, double tol_inner, int max_outer) {
  __shared__ double red[32];
  int active = 0;
  for (int s = threadIdx.x; s < b.nslots; s += blockDim.x) {
    if (b.outer_done[s]) continue;
    const JuncDev& J = jt[b.junc[s]];
    double nrm = 0.0;
    const double* np = b.nrm0_part + (size_t)s * b.PA;
    for (int t = 0; t < J.nR; ++t) nrm += np[t];
    const double rel = sqrt(nrm / b.bnorm2[s]);
    b.relres[s] = rel;
    if (rel <= tol) {
      b.outer_done[s] = 1;
      b.done[s] = 1;
    } else if (!isfinite(rel) || b.n_outer[s] >= max_outer || b.breakdowns[s] > max_outer) {
      b.outer_done[s] = 1;
      b.done[s] = 1;
      b.status[s] = (b.breakdowns[s] > 0 && b.n_outer[s] < max_outer) ? 2 : 1;
    } else {
      b.n_outer[s] += 1;
      b.iters[s] = 0;
      b.done[s] = 0;
      const double t_in = tol_inner * tol_inner * nrm;
      const double t_out = 0.25 * tol * tol * b.bnorm2[s];
      b.tol2[s] = t_in > t_out ? t_in : t_out;
    }
    active += b.outer_done[s] ? 0 : 1;
  }
  double v[1] = {(double)active};
  double out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) b.n_active[1] = (int)out[0];
}

// x64 += d, d = 0 for systems still being refined (runs between the true
// residual and the refinement bookkeeping, so it sees the previous outer_done
// flags; each thread touches only its own points).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) x_update_kernel(const JuncDev* __restrict__ jt, const BatchDev b) {
  using C = typename cx<T>::t;
  const int s = blockIdx.y;
  if (b.outer_done[s]) return;
  const JuncDev& J = jt[b.junc[s]];
  if ((int)blockIdx.x >= J.nB) return;
  const long long vo = b.voff[s];
  const long long i0 = (long long)blockIdx.x * kVecPts;
  const long long i1 = min(i0 + (long long)kVecPts, J.N);
  C* dv = reinterpret_cast<C*>(b.d);
  for (long long i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
    const double2 d = to64(dv[vo + i]);
    double2 x = b.x64[vo + i];
    x.x += d.x;
    x.y += d.y;
    b.x64[vo + i] = x;
    dv[vo + i] = czero<C>();
  }
}

// ||b||^2 of adjoint right-hand sides b = Gamma_L o conj(xf) (one CTA per slot).
__global__ void __launch_bounds__(256) bnorm_adjoint_kernel(const JuncDev* __restrict__ jt, const BatchDev b) {
  const int s = blockIdx.x;
  if (b.outer_done[s] || b.col[s] >= 0) return;
  const JuncDev& J = jt[b.junc[s]];
  __shared__ double red[32];
  const long long vo = b.voff[s];
  double acc = 0.0;
  for (int l = threadIdx.x; l < J.nL; l += blockDim.x) {
    const double g = J.L_gam[l];
    const double2 x = b.xf[vo + J.L_idx[l]];
    acc += g * g * (x.x * x.x + x.y * x.y);
  }
  double v[1] = {acc};
  double out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) b.bnorm2[s] = out[0] > 0.0 ? out[0] : 1.0;
}

// t_s = sum_{i in L} Gamma_L,i |x_s(i)|^2 (FP64, fixed order), written to
// t_out[out_index[s]] (slots with out_index < 0 are idle).
__global__ void __launch_bounds__(256) t_partial_kernel(const JuncDev* __restrict__ jt, const BatchDev b,
                                                        const int* __restrict__ out_index,
                                                        double* __restrict__ t_out) {
  const int s = blockIdx.x;
  const int o = out_index[s];
  if (o < 0) return;
  const JuncDev& J = jt[b.junc[s]];
  __shared__ double red[32];
  const long long vo = b.voff[s];
  double acc = 0.0;
  for (int l = threadIdx.x; l < J.nL; l += blockDim.x) {
    const double2 x = b.x64[vo + J.L_idx[l]];
    acc += J.L_gam[l] * (x.x * x.x + x.y * x.y);
  }
  double v[1] = {acc};
  double out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) t_out[o] = out[0];
}

// T[e] = 4 sum_c Gamma_R[cols[c]] t[e][c]   (one warp per energy, fixed order).
__global__ void t_final_kernel(int n_e, int n_cols, const double* __restrict__ t_all,
                               const double* __restrict__ gr_cols, double* __restrict__ T) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= n_e) return;
  double acc = 0.0;
  for (int c = lane; c < n_cols; c += 32) acc += gr_cols[c] * t_all[(size_t)e * n_cols + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) T[e] = 4.0 * acc;
}

// g[i] += sum_s wt[s] Re(lambda_s(i) x_s(i)), lambda in x64 (adjoint), x in xf.
__global__ void __launch_bounds__(256) grad_accum_kernel(const BatchDev b, long long N, const double* __restrict__ wt,
                                                         double* __restrict__ g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int s = 0; s < b.nslots; ++s) {
    const double w = wt[s];
    if (w == 0.0) continue;
    const long long gi = b.voff[s] + i;
    const double2 l = b.x64[gi];
    const double2 x = b.xf[gi];
    acc += w * (l.x * x.x - l.y * x.y);
  }
  g[i] += acc;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_op_R1(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev&,
                         const void*, void*, const void*);
cudaError_t launch_op_R2(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev&,
                         const void*, void*, const void*);
cudaError_t launch_op_R3(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev&,
                         const void*, void*, const void*);
cudaError_t launch_op_R4(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev&,
                         const void*, void*, const void*);
cudaError_t launch_op_R5(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev&,
                         const void*, void*, const void*);
cudaError_t launch_op_R6(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev&,
                         const void*, void*, const void*);

cudaError_t launch_op(int mode, bool fp32, int R, int ppt, dim3 grid, int threads, size_t smem, cudaStream_t st,
                      const JuncDev* jt, const BatchDev& b, const void* x_in, void* y_out, const void* c_in) {
  switch (R) {
    case 1: return launch_op_R1(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 2: return launch_op_R2(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 3: return launch_op_R3(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 4: return launch_op_R4(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 5: return launch_op_R5(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 6: return launch_op_R6(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    default: return cudaErrorInvalidValue;
  }
}

size_t op_smem_bytes(bool fp32, int mode, int R, int TY, int nx, int n_proj) {
  const size_t el = (mode == OP_RESID || !fp32) ? sizeof(double2) : sizeof(float2);
  return el * (2 * (size_t)(TY + 2 * R) * (nx + 2 * R) + (size_t)n_proj);
}

cudaError_t launch_cocg_update(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt,
                               const BatchDev& b) {
  dim3 grid(nB, nslots);
  if (fp32) cocg_update_kernel<float><<<grid, kVecThreads, 0, st>>>(jt, b);
  else cocg_update_kernel<double><<<grid, kVecThreads, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_project(int mode, bool fp32, int nslots, int n_groups, cudaStream_t st, const JuncDev* jt,
                           const BatchDev& b, const void* x_in, void* c_out) {
  dim3 grid(n_groups, nslots);
  if (mode == PJ_R) {
    if (fp32) project_kernel<float, PJ_R><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
    else project_kernel<double, PJ_R><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
  } else if (mode == PJ_X) {
    if (fp32) project_kernel<float, PJ_X><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
    else project_kernel<double, PJ_X><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
  } else {
    if (fp32) project_kernel<float, PJ_IN><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
    else project_kernel<double, PJ_IN><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_inner_book(int nslots, int max_iter, cudaStream_t st, const JuncDev* jt, const BatchDev& b) {
  (void)nslots;
  inner_book_kernel<<<1, 1024, 0, st>>>(jt, b, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_outer_book(int nslots, double tol, double tol_inner, int max_outer, cudaStream_t st,
                              const JuncDev* jt, const BatchDev& b) {
  (void)nslots;
  outer_book_kernel<<<1, 1024, 0, st>>>(jt, b, tol, tol_inner, max_outer);
  return cudaGetLastError();
}

cudaError_t launch_x_update(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt, const BatchDev& b) {
  dim3 grid(nB, nslots);
  if (fp32) x_update_kernel<float><<<grid, kVecThreads, 0, st>>>(jt, b);
  else x_update_kernel<double><<<grid, kVecThreads, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_bnorm_adjoint(int nslots, cudaStream_t st, const JuncDev* jt, const BatchDev& b) {
  bnorm_adjoint_kernel<<<nslots, 256, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_t_partial(int nslots, cudaStream_t st, const JuncDev* jt, const BatchDev& b,
                             const int* out_index, double* t_out) {
  t_partial_kernel<<<nslots, 256, 0, st>>>(jt, b, out_index, t_out);
  return cudaGetLastError();
}

cudaError_t launch_t_final(int n_e, int n_cols, cudaStream_t st, const double* t_all, const double* gr_cols,
                           double* T_out) {
  const int warps = 8;
  t_final_kernel<<<(n_e + warps - 1) / warps, 32 * warps, 0, st>>>(n_e, n_cols, t_all, gr_cols, T_out);
  return cudaGetLastError();
}

cudaError_t launch_grad_accum(int nslots, long long N, cudaStream_t st, const BatchDev& b, const double* wt,
                              double* g) {
  (void)nslots;
  grad_accum_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(b, N, wt, g);
  return cudaGetLastError();
}

}  // namespace rsn
