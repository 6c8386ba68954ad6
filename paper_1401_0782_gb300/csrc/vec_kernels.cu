// Streaming, reduction and scheduling kernels of the batched COCG solver,
// the T(E) reduction (Eq. T-realspace) and the adjoint gradient.
//
// Per iteration of the streaming solver (all kernels skip slots in other states):
//   zero      (NEW)            x = 0, d = 0
//   project   (NEW|CHECK)      c_x = v_p . (x + d)                       [projectors]
//   op RESID  (NEW|CHECK)      r = b - A (x + d) in FP64, ||r||^2, r^T r
//   x_update  (NEW|CHECK)      x += d, d = 0
//   sched     (all, 1 CTA)     converged? -> DRAIN; else reliable update -> ACTIVE;
//                              DRAIN -> FREE; FREE slots take queued systems
//   emit      (DRAIN)          T partial of the finished system
//   project   (ACTIVE)         c_r = v_p . r                             [projectors]
//   op COCG   (ACTIVE)         p = r + beta p, q = A p, p^T q
//   update    (ACTIVE)         alpha = rho/mu, r -= alpha q, d += alpha p, r^T r, ||r||^2
//   book      (ACTIVE, 1 CTA)  iteration counts; recurrence target reached -> CHECK
#include <algorithm>
#include <type_traits>

#include "cplx.cuh"
#include "ops_kernel.cuh"
#include "rsn_internal.h"

namespace rsn {

// ---------------------------------------------------------------------------
// List of the slots that need a true residual in this iteration (NEW and
// CHECK), in slot order: one CTA, ballot + warp-count prefix per 1024 slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSchedThreads) list_kernel(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  __shared__ int warp_cnt[kSchedThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int total = 0;
  for (int base = 0; base < b.nslots; base += blockDim.x) {
    const int s = base + threadIdx.x;
    int st = SL_FREE;
    if (s < b.nslots) st = b.state[s];
    const bool in = st == SL_NEW || st == SL_CHECK || st == SL_CHECKT;
    if (s < b.nslots) b.inlist[s] = in ? 1 : 0;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    int before = 0, sum = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += warp_cnt[w];
      sum += warp_cnt[w];
    }
    if (in) b.lst[total + before + __popc(m & ((1u << lane) - 1u))] = s;
    total += sum;
    __syncthreads();
  }
  if (threadIdx.x == 0) *b.lst_n = total;
}

// ---------------------------------------------------------------------------
// zero x and d of newly assigned systems (CTA rows over the NEW / CHECK list)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kVecThreads) zero_kernel(const JuncDev* __restrict__ jt,
                                                           const BatchDev* __restrict__ bp) {
  using C = typename cx<T>::t;
  const BatchDev& b = *bp;
  const int n = *b.lst_n;
  for (int li = blockIdx.y; li < n; li += gridDim.y) {
    const int s = b.lst[li];
    if (b.state[s] != SL_NEW) continue;
    const JuncDev& J = jt[b.junc[s]];
    if ((int)blockIdx.x >= J.nB) continue;
    const long long vo = b.voff[s], xo = b.xo[s];
    const long long i0 = (long long)blockIdx.x * kVecPts, i1 = min(i0 + (long long)kVecPts, J.N);
    C* dv = reinterpret_cast<C*>(b.d);
    const bool keep_x = b.warm[s] != 0;
    for (long long i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
      if (!keep_x) b.x64[xo + i] = make_double2(0.0, 0.0);
      dv[vo + i] = czero<C>();
    }
  }
}

// ---------------------------------------------------------------------------
// COCG update (after the operator kernel of the same iteration):
//   alpha = rho_k / mu_k,  r -= alpha q,  d += alpha p_new,
//   partial sums of rho_{k+1} = r^T r and ||r||^2.
// q arrives without the projector term (the operator kernel leaves it out);
// on the points inside a projector support the term -sum_p v_p(i) e_kb[p] c_p
// is added here, from e_kb c_p of the new direction (projection kernel, staged
// in shared memory with its zero-padded tail), so q is never written back.
// Each CTA covers kVecPts consecutive points of one system.  A non-finite
// alpha leaves r and d untouched and flags the slot through a NaN norm.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cocg_update_kernel(const JuncDev* __restrict__ jt,
                                                                  const BatchDev* __restrict__ bp) {
  using C = typename cx<T>::t;
  const BatchDev& b = *bp;
  const int s = blockIdx.y;
  if (b.state[s] != SL_ACTIVE) return;
  const JuncDev& J = jt[b.junc[s]];
  if ((int)blockIdx.x >= J.nB) return;
  __shared__ double red[32 * 3];
  __shared__ double2 s_mu[kVecThreads];
  __shared__ double2 s_alpha;
  extern __shared__ __align__(16) unsigned char upd_smem[];
  C* s_ce = reinterpret_cast<C*>(upd_smem);  // e_kb c_p of the new direction, ce_stride entries
  const int k = b.iters[s];
  const int np = J.n_proj;
  if (np > 0) {
    const C* cen = reinterpret_cast<const C*>(b.c_e) + (size_t)s * b.ce_stride;
    for (int p = threadIdx.x; p < b.ce_stride; p += kVecThreads) s_ce[p] = cen[p];
  }
  // mu = p^T A p from the operator kernel's partials (any number of tiles)
  // followed by one partial per atom from the projection kernel: thread t adds
  // partials t, t + 256, ... and thread 0 adds those sums in thread order, so
  // the order is fixed for a given tiling
  const int nA = J.nA + (J.n_proj > 0 ? J.n_groups : 0);
  {
    double2 m = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < nA; t += kVecThreads) {
      const double2 v = b.mu_part[(size_t)s * b.PA + t];
      m.x += v.x;
      m.y += v.y;
    }
    s_mu[threadIdx.x] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 mu = make_double2(0.0, 0.0);
    for (int t = 0; t < kVecThreads && t < nA; ++t) { mu.x += s_mu[t].x; mu.y += s_mu[t].y; }
    s_alpha = cdiv(b.rho_cur[s], mu);
  }
  __syncthreads();
  const double2 a64 = s_alpha;
  if (b.n_shift > 0 && blockIdx.x == 0 && threadIdx.x == 0) b.salpha[(size_t)(k & 1) * b.nslots + s] = a64;
  const size_t slot_out = (size_t)s * b.PB + blockIdx.x;
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
  const int nq = J.inv_nq;
  for (long long i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
    const long long g = vo + i;
    const C p = pn[g];
    C q = qv[g];
    if (np > 0) {
      const int e0 = J.inv_ptr[i], e1 = J.inv_ptr[i + 1];
      for (int e = e0; e < e1; ++e) {
        const C* cp = s_ce + J.inv_p0[e];
        for (int qd = 0; qd < nq; ++qd) q = proj_quad<C, T>(J, e * nq + qd, cp + 4 * qd, q);
      }
    }
    C r = rv[g];
    r.x -= alpha.x * q.x - alpha.y * q.y;
    r.y -= alpha.x * q.y + alpha.y * q.x;
    C d = dv[g];
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
// Projections c_p = v_p . v for every projector, one CTA per (atom, slot):
// the atom's support is gathered once and dotted with each of its projectors.
//   PJ_R: v = r (inner precision), ACTIVE slots         -> c_r
//   PJ_X: v = x64 + d (FP64), NEW / CHECK slots         -> c_x
//   PJ_IN: v = x_in (apply entry point)                 -> c_out
// ---------------------------------------------------------------------------
enum { PJ_R = 0, PJ_X = 1, PJ_IN = 2 };

template <typename T, int MODE, int NP, int SPB>
__global__ void __launch_bounds__(128) project_kernel(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp,
                                                      const void* __restrict__ x_in, void* __restrict__ c_out) {
  // NP: projectors per atom at compile time (>= the junction's largest group);
  // SPB: slots per CTA, so each projector value is loaded once for SPB slots
  using CT = typename std::conditional<MODE == PJ_X, double, T>::type;
  using C = typename cx<CT>::t;
  using CO = typename cx<T>::t;
  const BatchDev& b = *bp;
  const int g = blockIdx.x;
  __shared__ double red[32 * 2];
  __shared__ int s_slot[SPB];
  __shared__ int s_any;
  // PJ_X takes SPB entries of the NEW / CHECK list per CTA row (rows stride by
  // gridDim.y); PJ_R and PJ_IN take slots blockIdx.y * SPB + u
  int n_ent = b.nslots;
  if constexpr (MODE == PJ_X) n_ent = *b.lst_n;
  for (int base = blockIdx.y * SPB; base < n_ent; base += gridDim.y * SPB) {
    __syncthreads();  // s_slot, s_any and red of the previous entries are consumed
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (threadIdx.x < SPB) {
      const int e = base + threadIdx.x;
      int s = e;
      if constexpr (MODE == PJ_X) s = e < n_ent ? b.lst[e] : -1;
      bool use = s >= 0 && s < b.nslots;
      if (use) {
        if constexpr (MODE == PJ_R) {
          use = b.state[s] == SL_ACTIVE;
        } else if constexpr (MODE == PJ_X) {
          const int st = b.state[s];
          use = st == SL_NEW || st == SL_CHECK;
        }
      }
      if (use && g >= jt[b.junc[s]].n_groups) use = false;
      s_slot[threadIdx.x] = use ? s : -1;
      if (use) atomicOr(&s_any, 1);
    }
    __syncthreads();
    if (!s_any) continue;
    int slot[SPB];
    long long vo[SPB], xo[SPB];
    double sig[SPB];
#pragma unroll
    for (int u = 0; u < SPB; ++u) {
      slot[u] = s_slot[u];
      const int s = slot[u] >= 0 ? slot[u] : 0;
      vo[u] = b.voff[s];
      xo[u] = (MODE == PJ_X) ? b.xo[s] : 0;
      sig[u] = (MODE == PJ_X) ? b.sigma[s] : 1.0;
    }
    // every active slot of this CTA belongs to a junction with this group; the
    // junction of the first active slot supplies the support (batches share it)
    int s0 = 0;
    for (int u = 0; u < SPB; ++u)
      if (slot[u] >= 0) {
        s0 = slot[u];
        break;
      }
    const JuncDev& J = jt[b.junc[s0]];
    const int p0 = J.grp_p0[g], np = J.grp_np[g];
    const int k0 = J.grp_ptr[g], k1 = J.grp_ptr[g + 1], len = k1 - k0;
    const long long vb = J.grp_voff[g];
    C acc[SPB][NP];
#pragma unroll
    for (int u = 0; u < SPB; ++u)
#pragma unroll
      for (int p = 0; p < NP; ++p) acc[u][p] = czero<C>();
    for (int kk = k0 + threadIdx.x; kk < k1; kk += blockDim.x) {
      const int gi = J.grp_idx[kk];
      const long long vk = vb + (kk - k0);
      CT a[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (p < np) {
          if constexpr (sizeof(CT) == 8) a[p] = (CT)J.grp_val64[vk + (long long)p * len];
          else a[p] = (CT)J.grp_val32[vk + (long long)p * len];
        } else {
          a[p] = 0;
        }
      }
#pragma unroll
      for (int u = 0; u < SPB; ++u) {
        if (slot[u] < 0) continue;
        C v;
        if constexpr (MODE == PJ_R) {
          v = reinterpret_cast<const CO*>(b.r)[vo[u] + gi];
        } else if constexpr (MODE == PJ_X) {
          const double2 xx = b.x64[xo[u] + gi];
          const double2 dd = to64(reinterpret_cast<const CO*>(b.d)[vo[u] + gi]);
          v = mk2(fma(sig[u], dd.x, xx.x), fma(sig[u], dd.y, xx.y));
        } else {
          v = reinterpret_cast<const CO*>(x_in)[vo[u] + gi];
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[u][p] = rfma(a[p], v, acc[u][p]);
      }
    }
#pragma unroll
    for (int u = 0; u < SPB; ++u) {
      if (slot[u] < 0) continue;  // uniform across the CTA
      const int sl = slot[u];
      C* out = reinterpret_cast<C*>(c_out) + (size_t)sl * b.pstride + p0;
      // PJ_R, thread 0: the projections of the new direction
      // c_p = c_r + beta c_p_old (c_p = c_r in the first iteration), e_kb c_p
      // for the update kernel, and this atom's share of mu = p^T A p,
      // -sum_p e_kb[p] c_p^2, as one more partial after the operator tiles'
      double2 mu_g = make_double2(0.0, 0.0);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (p < np) {  // uniform across the CTA
          CT v[2] = {acc[u][p].x, acc[u][p].y};
          double o[2];
          block_sum<2>(v, red, o);
          if (threadIdx.x == 0) {
            const C cr = mk2((CT)o[0], (CT)o[1]);
            out[p] = cr;
            if constexpr (MODE == PJ_R) {
              const int k = b.iters[sl];
              const C* cpo = reinterpret_cast<const C*>(b.c_p) + ((size_t)(k & 1) * b.nslots + sl) * b.pstride;
              C* cpn = reinterpret_cast<C*>(b.c_p) + ((size_t)((k + 1) & 1) * b.nslots + sl) * b.pstride;
              C* cen = reinterpret_cast<C*>(b.c_e) + (size_t)sl * b.ce_stride;
              C c = cr;
              if (k > 0) c = cfma(from64<C>(b.beta_cur[sl]), cpo[p0 + p], c);
              cpn[p0 + p] = c;
              const CT e = (CT)J.ekb[p0 + p];
              cen[p0 + p] = mk2(e * c.x, e * c.y);
              const double cx = c.x, cy = c.y, e64 = J.ekb[p0 + p];
              mu_g.x -= e64 * (cx * cx - cy * cy);
              mu_g.y -= e64 * (2.0 * cx * cy);
            }
          }
        }
      }
      if (MODE == PJ_R && threadIdx.x == 0) b.mu_part[(size_t)sl * b.PA + J.nA + g] = mu_g;
    }
  }  // list entries
}

// ---------------------------------------------------------------------------
// Bookkeeping after each COCG iteration, one warp per slot: rho_{k+1} and
// ||r||^2 from the update kernel's partials (fixed-order warp tree),
// beta_{k+1} = rho_{k+1} / rho_k, iteration counts, the recurrence target of
// the current cycle, breakdown detection (NaN partial from the update kernel).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kBookWarps) book_kernel(const JuncDev* __restrict__ jt,
                                                              const BatchDev* __restrict__ bp, int slot_it) {
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * kBookWarps + (threadIdx.x >> 5);
  if (s >= b.nslots || b.state[s] != SL_ACTIVE) return;
  const JuncDev& J = jt[b.junc[s]];
  double nrm = 0.0, rx = 0.0, ry = 0.0;
  for (int t = lane; t < J.nB; t += 32) {
    nrm += b.nrm_part[(size_t)s * b.PB + t];
    const double2 v = b.rho_part[(size_t)s * b.PB + t];
    rx += v.x;
    ry += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    rx += __shfl_down_sync(0xffffffffu, rx, o);
    ry += __shfl_down_sync(0xffffffffu, ry, o);
  }
  if (lane != 0) return;
  const int k = b.iters[s] + 1;
  b.iters[s] = k;
  const int tot = b.total_iters[s] + 1;
  b.total_iters[s] = tot;
  const int cyc = b.cyc_iters[s] + 1;
  b.cyc_iters[s] = cyc;
  atomicAdd(b.counters, 1ull);
  atomicAdd(b.sched + 3 + kMaxGraphIters + slot_it, 1);
  const double2 rho = make_double2(rx, ry);
  if (b.n_shift > 0) b.rn2[s] = nrm;
  b.beta_cur[s] = cdiv(rho, b.rho_cur[s]);
  b.rho_cur[s] = rho;
  if (!isfinite(nrm)) {
    b.restart[s] = 1;
    b.rrec2[s] = 0.0;
    b.state[s] = SL_CHECK;
  } else if (nrm <= b.tol2[s] || tot >= b.max_iter || cyc >= b.cycle_cap) {
    b.rrec2[s] = nrm;
    b.state[s] = b.gphase[s] ? SL_CHECKT : SL_CHECK;
  }
}

// ---------------------------------------------------------------------------
// Scheduler (one CTA, after the true-residual path and the COCG step of the
// same iteration): finishes converged
// systems, performs reliable updates (the true FP64 residual replaces the
// recurrence residual, the search direction is kept), frees drained slots and
// assigns queued systems to free slots in slot order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSchedThreads) sched_kernel(const JuncDev* __restrict__ jt,
                                                             const BatchDev* __restrict__ bp, int slot_it) {
  const BatchDev& b = *bp;
  const int S = b.nslots;
  __shared__ int warp_cnt[32];
  __shared__ double red[32 * 2];
  int upd = 0, busy = 0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    int st = b.state[s];
    // NEW / CHECK / CHECKT slots are handled only if this iteration's list took
    // them (their true residual or goal check ran): the bookkeeping kernel, which
    // runs beside the list path, can move a slot to CHECK after the list was made
    const bool listed = b.inlist[s] != 0;
    if (st == SL_DRAIN) {
      st = SL_FREE;
    } else if (st == SL_CHECKT && listed) {
      // goal phase: compare the T partial of the iterate with the previous check;
      // the recurrence continues untouched towards a tenfold lower residual
      const double tcur = b.tgoal[s], tl = b.tlast[s];
      b.tlast[s] = tcur;
      const int gcnt = b.gcnt[s] + 1;
      b.gcnt[s] = gcnt;
      const bool settled = fabs(tcur - tl) <= b.tol_T * fabs(tcur);
      const bool capped = gcnt >= kMaxGoalChecks || b.total_iters[s] >= b.max_iter;
      if (settled || capped) {
        // a mixed-precision system whose T partial did not settle within the cap
        // is handed back (solved again in FP64); FP64 keeps its iterate
        const bool back = !settled && b.handback;
        const int sy = b.sys[s];
        b.out_iters[sy] = b.total_iters[s];
        b.out_relres[sy] = b.rgoal[s];
        b.out_status[sy] = back ? 3 : 0;
        atomicAdd(b.counters + 2, 1ull);
        if (back) atomicAdd(b.counters + 3, 1ull);
        st = SL_DRAIN;
      } else {
        b.tol2[s] = 0.01 * b.rrec2[s];
        b.cyc_iters[s] = 0;
        st = SL_ACTIVE;
      }
    } else if ((st == SL_NEW || st == SL_CHECK) && listed) {
      const JuncDev& J = jt[b.junc[s]];
      double nrm = 0.0, tcur = 0.0;
      double2 rho = make_double2(0.0, 0.0);
      const double* np = b.nrm0_part + (size_t)s * b.PA;
      const double* tp = b.t0_part + (size_t)s * b.PA;
      const double2* rp = b.rho0_part + (size_t)s * b.PA;
      for (int t = 0; t < J.nR; ++t) {
        nrm += np[t];
        tcur += tp[t];
        rho.x += rp[t].x;
        rho.y += rp[t].y;
      }
      if (st == SL_NEW) {
        // cold start: r = b, so ||b||^2 = nrm; warm start: ||b||^2 is given
        const double bn = b.warm[s] ? b.sys_bn2[b.sys[s]] : nrm;
        b.bnorm2[s] = bn > 0.0 ? bn : 1.0;
        b.sigma[s] = bn > 0.0 ? sqrt(bn) : 1.0;
        b.rlast2[s] = 4.0 * nrm;
        b.stall[s] = 0;
        b.iters[s] = 0;
        b.total_iters[s] = 0;
        b.n_upd[s] = 0;
        b.restart[s] = 0;
        b.tlast[s] = -1.0;
        b.gcnt[s] = 0;
        b.gphase[s] = 0;
      }
      const double bn2 = b.bnorm2[s];
      const double rel = sqrt(nrm / bn2);
      const int sy = b.sys[s];
      const double tol = b.col[s] >= 0 ? b.tol : b.tol_adj;
      // a shifted system reaches CHECK only once every shift converged (or at
      // the iteration cap, which its per-shift records show): it is finished
      const bool res_ok = ((st == SL_CHECK || b.warm[s]) && rel <= tol) || nrm == 0.0;
      // goal-oriented finish of forward systems: the transmission reads x only
      // on the Gamma_L support, where x is exponentially small when the lead
      // channels are closed, so a residual of tol relative to the whole column
      // does not fix it; once the residual meets tol, iterations continue until
      // sum Gamma_L |x|^2 changes by at most tol_T of itself between two true
      // residuals (the Krylov iterate keeps converging there after its residual
      // has reached the rounding floor)
      const double tl = b.tlast[s];
      b.tlast[s] = tcur;
      const bool goal = b.tol_T > 0.0 && b.col[s] >= 0 && b.n_shift == 0;
      const bool goal_ok = !goal || nrm == 0.0 || (tl >= 0.0 && fabs(tcur - tl) <= b.tol_T * fabs(tcur));
      const bool goal_phase = res_ok && !goal_ok;  // the residual met tol, the T partial not yet
      // a goal phase that would start at the iteration or update cap keeps its
      // residual-converged iterate
      const bool goal_capped = goal_phase && (b.total_iters[s] >= b.max_iter || b.n_upd[s] >= b.max_upd);
      const bool conv = (res_ok && goal_ok) || goal_capped || (b.n_shift > 0 && st == SL_CHECK);
      // the recurrence has drifted when the true residual is more than 4x the
      // recurrence residual of the cycle that just ended (rounding in the
      // inner-precision Krylov basis): restart it from the true residual.
      // Cycles that did not cut the previous true residual by 4x are counted.
      // Early on such a plateau is ordinary slow Krylov convergence on an
      // indefinite operator, and a restart would throw the Krylov space away;
      // within three decades of the tolerance, two of them in a row mean the
      // recurrence has lost its accuracy (the true residuals that replace it
      // at the cycle cap hide the drift) and it restarts.
      // (in the goal phase the residual sits at its rounding floor: neither applies)
      const bool drift = st == SL_CHECK && !goal_phase && nrm > 16.0 * b.rrec2[s] * bn2;
      const bool no_gain = st == SL_CHECK && !goal_phase && nrm > 0.0625 * b.rlast2[s];
      const int stall = no_gain ? b.stall[s] + 1 : 0;
      // precision-limited systems are handed back early: either the true
      // residual stopped improving, or its rate so far (log rel per
      // iteration) predicts more iterations than the budget allows
      const int tot = b.total_iters[s];
      const bool slow = st == SL_CHECK && !goal_phase && tot >= 500 &&
                        (rel >= 1.0 || (double)tot * log(tol) / log(rel) > 1.5 * (double)b.max_iter);
      const bool stalled = (b.stall_cap > 0 && stall >= b.stall_cap) || (b.handback && slow);
      const bool fail = !isfinite(rel) || b.total_iters[s] >= b.max_iter || b.n_upd[s] >= b.max_upd || stalled;
      if (conv || fail) {
        b.out_iters[sy] = b.total_iters[s];
        b.out_relres[sy] = rel;
        b.out_status[sy] = conv ? 0 : (stalled ? 3 : (b.restart[s] ? 2 : 1));
        atomicAdd(b.counters + 2, 1ull);               // finished systems
        if (!conv) atomicAdd(b.counters + 3, 1ull);    // handed back (precision-limited / failed)
        st = SL_DRAIN;
      } else {
        // a drifted recurrence restarts from the true residual instead of
        // continuing with its direction
        b.stall[s] = stall;
        if (drift || (stall >= 2 && rel < 1e3 * tol)) b.restart[s] = 1;
        const double2 rho_s = make_double2(rho.x / bn2, rho.y / bn2);  // r^T r of r / sigma
        b.rlast2[s] = nrm;
        if (st == SL_NEW || b.restart[s]) {
          // fresh start: p = r at the next iteration
          b.iters[s] = 0;
          b.restart[s] = 0;
        } else {
          // reliable update: the true residual replaces the recurrence residual
          // and the direction update continues with beta_k = rho_new / rho_{k-1}
          // (beta_cur holds rho_k / rho_{k-1}, rho_cur holds rho_k)
          b.beta_cur[s] = cmul(b.beta_cur[s], cdiv(rho_s, b.rho_cur[s]));
        }
        b.rho_cur[s] = rho_s;
        // targets in the inner vectors' units (r / sigma, sigma^2 = ||b||^2)
        const double t_in = b.delta * b.delta * nrm / bn2, t_out = 0.25 * tol * tol;
        // shifted systems: the shift kernel ends the cycle once every shift converged;
        // goal phase: cycles of a tenfold cut of the recurrence residual
        b.tol2[s] = b.n_shift > 0 ? 0.0 : goal_phase ? 0.01 * nrm / bn2 : (t_in > t_out ? t_in : t_out);
        if (goal_phase) {
          // from here on the T partial is checked without true residuals (CHECKT)
          b.gphase[s] = 1;
          b.rgoal[s] = rel;
          b.gcnt[s] = 0;
        }
        if (st == SL_CHECK) {
          b.n_upd[s] += 1;
          ++upd;
        }
        b.cyc_iters[s] = 0;
        st = SL_ACTIVE;
      }
    }
    b.state[s] = st;
  }
  __syncthreads();
  // Assign ready systems to FREE slots.  Free slots are taken in slot order,
  // systems in queue order from the first unstarted one, skipping those whose
  // dependency has not finished: an adjoint waits for its forward column but
  // does not hold up the systems queued behind it.  At most kReadyWindow
  // systems past the first unstarted one are examined.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  __shared__ int s_nf, s_done, s_first;
  // (1) the free slots, compacted in slot order
  if (threadIdx.x == 0) s_nf = 0;
  __syncthreads();
  for (int base = 0; base < S; base += blockDim.x) {
    const int s = base + threadIdx.x;
    const bool fr = s < S && b.state[s] == SL_FREE;
    const unsigned m = __ballot_sync(0xffffffffu, fr);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += warp_cnt[w];
      total += warp_cnt[w];
    }
    if (fr) b.fslot[s_nf + before + __popc(m & below)] = s;
    __syncthreads();
    if (threadIdx.x == 0) s_nf += total;
    __syncthreads();
  }
  const int nf = s_nf;
  const int next0 = b.sched[0];
  // (2) ready systems, in queue order, to the free slots
  if (threadIdx.x == 0) s_done = 0;
  __syncthreads();
  const int wend = min(b.nsys, next0 + kReadyWindow);
  for (int base = next0; base < wend && nf > 0; base += blockDim.x) {
    if (s_done >= nf) break;  // uniform: written before the last barrier
    const int n = base + threadIdx.x;
    bool ready = false;
    if (n < wend && !b.sys_started[n]) {
      const int dep = b.sys_dep ? b.sys_dep[n] : -1;
      ready = dep < 0 || b.out_status[dep] >= 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, ready);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += warp_cnt[w];
      total += warp_cnt[w];
    }
    const int k = s_done + before + __popc(m & below);
    if (ready && k < nf) {
      const int s = b.fslot[k];
      b.sys[s] = n;
      b.junc[s] = b.sys_junc[n];
      b.E[s] = b.sys_E[n];
      b.col[s] = b.sys_col[n];
      const long long xo = b.sys_xo[n];
      b.xo[s] = xo >= 0 ? xo : b.voff[s];
      b.xfo[s] = b.sys_xfo[n];
      b.warm[s] = (b.sys_bn2 != nullptr && b.sys_bn2[n] > 0.0) ? 1 : 0;
      b.state[s] = SL_NEW;
      b.sys_started[n] = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_done = min(nf, s_done + total);
    __syncthreads();
  }
  // (3) the first unstarted system
  if (threadIdx.x == 0) s_first = b.nsys;
  __syncthreads();
  for (int base = next0; base < b.nsys; base += blockDim.x) {
    const int n = base + threadIdx.x;
    if (n < b.nsys && !b.sys_started[n]) atomicMin(&s_first, n);
    __syncthreads();
    const bool found = s_first < b.nsys;
    __syncthreads();
    if (found) break;
  }
  for (int s = threadIdx.x; s < S; s += blockDim.x) busy += (b.state[s] != SL_FREE) ? 1 : 0;
  double v[2] = {(double)busy, (double)upd};
  double out[2];
  block_sum<2>(v, red, out);
  if (threadIdx.x == 0) {
    b.sched[0] = s_first;
    b.sched[1] = (int)out[0];
    b.sched[3 + slot_it] = (int)out[0];
    b.counters[1] += (unsigned long long)out[1];
  }
}

// After a true residual (NEW or CHECK slots): x64 += sigma d, d = 0, and the
// inner-precision residual is rescaled to r / sigma, sigma = ||b||, so the
// inner recurrence works on O(1) numbers whatever the size of b (an adjoint
// right-hand side Gamma_L o conj(x) can be ~1e-6 or smaller, whose squares
// would leave the FP32 range).  For a NEW slot sigma comes from the residual
// partials (r = b there); each thread touches only its own points.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) x_update_kernel(const JuncDev* __restrict__ jt,
                                                               const BatchDev* __restrict__ bp) {
  using C = typename cx<T>::t;
  const BatchDev& b = *bp;
  __shared__ double s_part[kVecThreads];
  __shared__ double s_sig;
  const int n = *b.lst_n;
  for (int li = blockIdx.y; li < n; li += gridDim.y) {
    const int s = b.lst[li];
    const int st = b.state[s];
    if (st != SL_NEW && st != SL_CHECK && st != SL_CHECKT) continue;
    const JuncDev& J = jt[b.junc[s]];
    if ((int)blockIdx.x >= J.nB) continue;
    __syncthreads();  // s_part / s_sig of the previous entry are consumed
    if (st == SL_NEW) {
      // ||b||^2 from the residual kernel's partials, in the fixed order of the
      // update kernel's mu sum
      double n2t = 0.0;
      for (int t = threadIdx.x; t < J.nR; t += kVecThreads) n2t += b.nrm0_part[(size_t)s * b.PA + t];
      s_part[threadIdx.x] = n2t;
      __syncthreads();
      if (threadIdx.x == 0) {
        double n2 = 0.0;
        for (int t = 0; t < kVecThreads && t < J.nR; ++t) n2 += s_part[t];
        s_sig = n2 > 0.0 ? sqrt(n2) : 1.0;
        if (blockIdx.x == 0) b.sigma[s] = s_sig;
      }
    } else if (threadIdx.x == 0) {
      s_sig = b.sigma[s];
    }
    __syncthreads();
    const double sig = s_sig;
    // a goal-phase check keeps the recurrence (r is not a fresh true residual)
    const T isig = st == SL_CHECKT ? (T)1 : (T)(1.0 / sig);
    const long long vo = b.voff[s], xo = b.xo[s];
    const long long i0 = (long long)blockIdx.x * kVecPts;
    const long long i1 = min(i0 + (long long)kVecPts, J.N);
    C* dv = reinterpret_cast<C*>(b.d);
    C* rv = reinterpret_cast<C*>(b.r);
    for (long long i = i0 + threadIdx.x; i < i1; i += kVecThreads) {
      const double2 d = to64(dv[vo + i]);
      double2 x = b.x64[xo + i];
      x.x = fma(sig, d.x, x.x);
      x.y = fma(sig, d.y, x.y);
      b.x64[xo + i] = x;
      dv[vo + i] = czero<C>();
      C r = rv[vo + i];
      r.x *= isig;
      r.y *= isig;
      rv[vo + i] = r;
    }
  }
}

// Goal-phase checks (CHECKT slots of the list, after x_update moved d into x):
// tgoal[s] = sum_{i in L} Gamma_L,i |x(i)|^2, one CTA per list entry.
__global__ void __launch_bounds__(256) tgoal_kernel(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  __shared__ double red[32];
  const int n = *b.lst_n;
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    const int s = b.lst[li];
    if (b.state[s] != SL_CHECKT) continue;  // uniform across the CTA
    const JuncDev& J = jt[b.junc[s]];
    const long long xo = b.xo[s];
    double acc = 0.0;
    for (int l = threadIdx.x; l < J.nL; l += blockDim.x) {
      const double2 x = b.x64[xo + J.L_idx[l]];
      acc += J.L_gam[l] * (x.x * x.x + x.y * x.y);
    }
    double v[1] = {acc};
    double out[1];
    block_sum<1>(v, red, out);
    if (threadIdx.x == 0) b.tgoal[s] = out[0];
  }
}

// T partial of finished forward systems: out_t[sys] = sum_{i in L} Gamma_L,i |x(i)|^2.
__global__ void __launch_bounds__(256) emit_kernel(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  const int s = blockIdx.x;
  if (b.state[s] != SL_DRAIN || b.out_t == nullptr || b.col[s] < 0) return;
  const JuncDev& J = jt[b.junc[s]];
  __shared__ double red[32];
  const long long xo = b.xo[s];
  double acc = 0.0;
  for (int l = threadIdx.x; l < J.nL; l += blockDim.x) {
    const double2 x = b.x64[xo + J.L_idx[l]];
    acc += J.L_gam[l] * (x.x * x.x + x.y * x.y);
  }
  double v[1] = {acc};
  double out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) b.out_t[b.sys[s]] = out[0];
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

// g[i] += sum_k wt[k] Re(lambda_k(i) x_k(i)) over systems k in index order
// (lambda_k = lam + k N, x_k = x + k N).
__global__ void __launch_bounds__(256) grad_sys_kernel(int nsys, long long N, const double2* __restrict__ lam,
                                                       const double2* __restrict__ x, const double* __restrict__ wt,
                                                       double* __restrict__ g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int k = 0; k < nsys; ++k) {
    const double w = wt[k];
    if (w == 0.0) continue;
    const double2 l = lam[(long long)k * N + i];
    const double2 v = x[(long long)k * N + i];
    acc += w * (l.x * v.x - l.y * v.y);
  }
  g[i] += acc;
}

// ---------------------------------------------------------------------------
// Shifted COCG (one seed Krylov space for every energy of a window).
//
// A(E_e) = A(E_s) + sigma_e 1 with sigma_e = E_e - E_s (Eq. G: E enters A only
// on the diagonal), so the seed recurrence's residual r_k = R_k(A_s) b serves
// every shifted system: its residual is collinear, r_{e,k} = r_k / pi_{e,k},
// with pi_{e,k} = R_k(-sigma_e) from the three-term recurrence of R_k:
//   pi_{k+1} = (1 + alpha_k sigma) pi_k + (alpha_k beta_{k-1} / alpha_{k-1}) (pi_k - pi_{k-1}),
//   alpha_e = alpha_k pi_k / pi_{k+1},  beta_e = beta_k (pi_k / pi_{k+1})^2,
//   x_e += alpha_e p_e,  p_e = r_{k+1} / pi_{k+1} + beta_e p_e
// (alpha_{-1} = 1, beta_{-1} = 0, pi_{-1} = pi_0 = 1, p_{e,0} = b).  The seed
// runs the FP64 slot solver unchanged; the shifted iterates live only on the
// tracked points (the Gamma_L support for T, every point for full columns).
// A shift is frozen once ||r_{k+1}|| / |pi_{e,k+1}| <= tol ||b||.
// ---------------------------------------------------------------------------

// x_e = 0, p_e = b on the tracked points, pi = 1, no shift converged; NEW slots
// (rows over the NEW / CHECK list, like the zero kernel)
__global__ void __launch_bounds__(kVecThreads) shift_init_kernel(const JuncDev* __restrict__ jt,
                                                                 const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  const int n = *b.lst_n, ns = b.n_shift, nT = b.nT;
  for (int li = blockIdx.y; li < n; li += gridDim.y) {
    const int s = b.lst[li];
    if (b.state[s] != SL_NEW) continue;
    const int col = b.col[s];
    double2* xb = b.xs + (long long)(b.xs_by_sys ? b.sys[s] : s) * b.xs_sstride;
    double2* pb = b.ps + (size_t)s * ns * nT;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nT; i += gridDim.x * blockDim.x) {
      const double one = b.T_idx[i] == col ? 1.0 : 0.0;
      for (int e = 0; e < ns; ++e) {
        xb[(long long)e * b.xs_estride + i] = make_double2(0.0, 0.0);
        pb[(size_t)e * nT + i] = make_double2(one, 0.0);
      }
    }
    if (blockIdx.x == 0) {
      const size_t S = (size_t)b.nslots;
      for (int e = threadIdx.x; e < ns; e += blockDim.x) {
        b.spi[(0 * S + s) * ns + e] = make_double2(1.0, 0.0);  // pi_0
        b.spi[(2 * S + s) * ns + e] = make_double2(1.0, 0.0);  // pi_{-1}
        b.sconv_it[(size_t)s * ns + e] = 0x7fffffff;
      }
      if (threadIdx.x == 0) {
        b.salpha[1 * S + s] = make_double2(1.0, 0.0);  // alpha_{-1}
        b.sbeta[1 * S + s] = make_double2(0.0, 0.0);   // beta_{-1}
      }
    }
  }
}

// One shifted step after iteration k of the seed (ACTIVE slots, and slots the
// bookkeeping kernel just moved to CHECK).  Every CTA of a slot derives the
// same scalars; CTA 0 records them (pi in a ring of three, so no CTA reads a
// value that is being overwritten) and ends the cycle once every shift converged.
__global__ void __launch_bounds__(kVecThreads) shift_update_kernel(const JuncDev* __restrict__ jt,
                                                                   const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  const int s = blockIdx.y;
  const int st = b.state[s];
  if (st != SL_ACTIVE && st != SL_CHECK) return;
  const int ns = b.n_shift, nT = b.nT;
  const size_t S = (size_t)b.nslots;
  const int k = b.iters[s] - 1;  // the iteration just completed
  extern __shared__ double2 sh[];  // [ns] alpha_e, [ns] beta_e, [ns] 1 / pi_{k+1}
  __shared__ int s_left;
  double2* sa = sh;
  double2* sb = sh + ns;
  double2* sip = sh + 2 * ns;
  if (threadIdx.x == 0) s_left = 0;
  __syncthreads();
  const double2 al = b.salpha[(size_t)(k & 1) * S + s];
  const double2 al_m = b.salpha[(size_t)((k + 1) & 1) * S + s];
  const double2 be = b.beta_cur[s];
  const double2 be_m = b.sbeta[(size_t)((k + 1) & 1) * S + s];
  const double rn2 = b.rn2[s], bn2 = b.bnorm2[s];
  const double2 cc = cmul(al, cdiv(be_m, al_m));  // alpha_k beta_{k-1} / alpha_{k-1}
  const double2* pi_k = b.spi + ((size_t)(k % 3) * S + s) * ns;
  const double2* pi_m = b.spi + ((size_t)((k + 2) % 3) * S + s) * ns;
  double2* pi_n = b.spi + ((size_t)((k + 1) % 3) * S + s) * ns;
  int* cit = b.sconv_it + (size_t)s * ns;
  for (int e = threadIdx.x; e < ns; e += blockDim.x) {
    if (cit[e] < k) {  // frozen at an earlier iteration
      sa[e] = make_double2(0.0, 0.0);
      sb[e] = make_double2(0.0, 0.0);
      sip[e] = make_double2(0.0, 0.0);
      continue;
    }
    const double sg = b.shift_sig[e];
    const double2 p0 = pi_k[e], pm = pi_m[e];
    // pi_{k+1} = (1 + alpha sigma) pi_k + c (pi_k - pi_{k-1})
    const double2 f = make_double2(1.0 + al.x * sg, al.y * sg);
    const double2 pn = cadd(cmul(f, p0), cmul(cc, csub(p0, pm)));
    const double2 ratio = cdiv(p0, pn);
    sa[e] = cmul(al, ratio);
    sb[e] = cmul(be, cmul(ratio, ratio));
    sip[e] = cdiv(make_double2(1.0, 0.0), pn);
    const double apn2 = pn.x * pn.x + pn.y * pn.y;
    const double est2 = rn2 / (apn2 * bn2);
    const bool conv = est2 <= b.tol * b.tol;
    if (!isfinite(est2)) sip[e] = make_double2(0.0, 0.0);
    if (blockIdx.x == 0) {
      pi_n[e] = pn;
      const int sy = b.sys[s];
      b.out_srel[(size_t)e * b.nsys + sy] = sqrt(est2);
      if (conv) {
        cit[e] = k;
        b.out_sit[(size_t)e * b.nsys + sy] = k + 1;
      } else {
        atomicAdd(&s_left, 1);
      }
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.sbeta[(size_t)(k & 1) * S + s] = be;
    if (s_left == 0) b.state[s] = SL_CHECK;  // every shift converged: end of the seed's cycle
  }
  double2* xb = b.xs + (long long)(b.xs_by_sys ? b.sys[s] : s) * b.xs_sstride;
  double2* pb = b.ps + (size_t)s * ns * nT;
  const double2* rv = reinterpret_cast<const double2*>(b.r) + b.voff[s];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nT; i += gridDim.x * blockDim.x) {
    const double2 r = rv[b.T_idx[i]];
    for (int e = 0; e < ns; ++e) {
      const double2 ip = sip[e];
      if (ip.x == 0.0 && ip.y == 0.0) continue;  // frozen (uniform across the CTA)
      double2* xp = xb + (long long)e * b.xs_estride + i;
      double2* pp = pb + (size_t)e * nT + i;
      const double2 p = *pp;
      *xp = cfma(sa[e], p, *xp);
      *pp = cfma(sb[e], p, cmul(r, ip));
    }
  }
}

// T partials of finished shifted systems: out_ts[e][sys] = sum over the tracked
// points of Gamma_L |x_e|^2 (one CTA per (shift, slot), fixed-order sums).
__global__ void __launch_bounds__(256) shift_emit_kernel(const JuncDev* __restrict__ jt,
                                                         const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  const int s = blockIdx.y, e = blockIdx.x;
  if (b.state[s] != SL_DRAIN || e >= b.n_shift) return;
  const JuncDev& J = jt[b.junc[s]];
  __shared__ double red[32];
  const double2* xb = b.xs + (long long)(b.xs_by_sys ? b.sys[s] : s) * b.xs_sstride + (long long)e * b.xs_estride;
  double acc = 0.0;
  for (int i = threadIdx.x; i < b.nT; i += blockDim.x) {
    const double g = J.gl[b.T_idx[i]];
    if (g > 0.0) {
      const double2 x = xb[i];
      acc += g * (x.x * x.x + x.y * x.y);
    }
  }
  double v[1] = {acc};
  double out[1];
  block_sum<1>(v, red, out);
  if (threadIdx.x == 0) b.out_ts[(size_t)e * b.nsys + b.sys[s]] = out[0];
}

// ---------------------------------------------------------------------------
// Landauer current (Eq. Landauer): I(V_k) = (2e/h) int T(E) [f(E - mu_L) -
// f(E - mu_R)] dE with mu_{L,R} = E_F +- V_k / 2, atomic units (2e/h = 1/pi),
// by the trapezoidal rule on the given ascending energy grid; one CTA per
// bias, fixed-order sums.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fermi_dev(double x, double kT) {
  if (kT == 0.0) return x < 0.0 ? 1.0 : (x > 0.0 ? 0.0 : 0.5);
  return 0.5 * (1.0 - tanh(x / (2.0 * kT)));
}

__global__ void __launch_bounds__(256) landauer_kernel(int n_e, const double* __restrict__ E,
                                                       const double* __restrict__ T, const double* __restrict__ V,
                                                       double E_F, double kT, double* __restrict__ I) {
  __shared__ double red[32];
  const double v = V[blockIdx.x];
  const double muL = E_F + 0.5 * v, muR = E_F - 0.5 * v;
  double acc = 0.0;
  for (int e = threadIdx.x; e + 1 < n_e; e += blockDim.x) {
    const double g0 = T[e] * (fermi_dev(E[e] - muL, kT) - fermi_dev(E[e] - muR, kT));
    const double g1 = T[e + 1] * (fermi_dev(E[e + 1] - muL, kT) - fermi_dev(E[e + 1] - muR, kT));
    acc += 0.5 * (E[e + 1] - E[e]) * (g0 + g1);
  }
  double vv[1] = {acc};
  double out[1];
  block_sum<1>(vv, red, out);
  if (threadIdx.x == 0) I[blockIdx.x] = out[0] / 3.14159265358979323846;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define RSN_DECL_OP(R)                                                                                        \
  cudaError_t launch_op_R##R(int, bool, int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev*, \
                             const void*, void*, const void*);                                                 \
  cudaError_t launch_op_tma_R##R(int, bool, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev*,  \
                                 const void*, void*, const void*);                                             \
  cudaError_t launch_op_pair_R##R(int, bool, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev*, \
                                  const void*, void*, const void*);                                            \
  cudaError_t launch_op_plane_R##R(int, dim3, int, size_t, cudaStream_t, const JuncDev*, const BatchDev*,      \
                                   const void*, void*, const void*);
RSN_DECL_OP(1)
RSN_DECL_OP(2)
RSN_DECL_OP(3)
RSN_DECL_OP(4)
RSN_DECL_OP(5)
RSN_DECL_OP(6)
#undef RSN_DECL_OP

cudaError_t launch_op(int mode, bool fp32, int R, int ppt, dim3 grid, int threads, size_t smem, cudaStream_t st,
                      const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
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

cudaError_t launch_op_tma(int mode, bool fp32, int R, dim3 grid, int threads, size_t smem, cudaStream_t st,
                          const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  switch (R) {
    case 1: return launch_op_tma_R1(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 2: return launch_op_tma_R2(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 3: return launch_op_tma_R3(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 4: return launch_op_tma_R4(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 5: return launch_op_tma_R5(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 6: return launch_op_tma_R6(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_op_pair(int mode, int R, bool big, dim3 grid, int threads, size_t smem, cudaStream_t st,
                           const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  switch (R) {
    case 1: return launch_op_pair_R1(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 2: return launch_op_pair_R2(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 3: return launch_op_pair_R3(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 4: return launch_op_pair_R4(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 5: return launch_op_pair_R5(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 6: return launch_op_pair_R6(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_op_plane(int mode, int R, dim3 grid, int threads, size_t smem, cudaStream_t st, const JuncDev* jt,
                            const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  switch (R) {
    case 1: return launch_op_plane_R1(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 2: return launch_op_plane_R2(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 3: return launch_op_plane_R3(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 4: return launch_op_plane_R4(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 5: return launch_op_plane_R5(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    case 6: return launch_op_plane_R6(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);
    default: return cudaErrorInvalidValue;
  }
}

size_t op_pair_smem_bytes(int mode, int R, int nx, int ny, int n_proj) {
  const size_t nin = mode == OP_COCG ? 2 : 1;
  const size_t pitch = (size_t)nx + 2 * kPairXO;
  const size_t cep = mode == OP_APPLY ? (size_t)n_proj + kCePad : 0;
  return sizeof(float2) * (kPairStages * nin * (size_t)nx * ny + 2 * (size_t)(ny + 2 * R) * pitch + cep) + 16 +
         8 * kPairStages;
}

size_t op_tma_smem_bytes(bool fp32, int mode, int R, int nx, int ny, int n_proj) {
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  const size_t nin = mode == OP_COCG ? 2 : 1;
  return el * (kStages * nin * (size_t)nx * ny + 2 * (size_t)(nx + 2 * R) * (ny + 2 * R) + (size_t)n_proj + kCePad) +
         16 + 8 * kStages;
}

size_t op_smem_bytes(bool fp32, int mode, int R, int TY, int nx, int n_proj) {
  const size_t el = (mode == OP_RESID || !fp32) ? sizeof(double2) : sizeof(float2);
  return el * (2 * (size_t)(TY + 2 * R) * (nx + 2 * R) + (size_t)n_proj + kCePad);
}

cudaError_t launch_zero(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  dim3 grid(nB, nslots);
  if (fp32) zero_kernel<float><<<grid, kVecThreads, 0, st>>>(jt, b);
  else zero_kernel<double><<<grid, kVecThreads, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_cocg_update(bool fp32, int nslots, int nB, int ce_stride, cudaStream_t st, const JuncDev* jt,
                               const BatchDev* b) {
  dim3 grid(nB, nslots);
  const size_t smem = (size_t)ce_stride * (fp32 ? sizeof(float2) : sizeof(double2));
  if (smem > 48 * 1024) {
    cudaError_t e = set_max_dynamic_smem(
        fp32 ? reinterpret_cast<const void*>(cocg_update_kernel<float>) : reinterpret_cast<const void*>(cocg_update_kernel<double>),
        smem);
    if (e != cudaSuccess) return e;
  }
  if (fp32) cocg_update_kernel<float><<<grid, kVecThreads, smem, st>>>(jt, b);
  else cocg_update_kernel<double><<<grid, kVecThreads, smem, st>>>(jt, b);
  return cudaGetLastError();
}

template <int NP, int SPB>
static void launch_project_np(int mode, bool fp32, dim3 grid, cudaStream_t st, const JuncDev* jt, const BatchDev* b,
                              const void* x_in, void* c_out) {
  if (mode == PJ_R) {
    if (fp32) project_kernel<float, PJ_R, NP, SPB><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
    else project_kernel<double, PJ_R, NP, SPB><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
  } else if (mode == PJ_X) {
    if (fp32) project_kernel<float, PJ_X, NP, SPB><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
    else project_kernel<double, PJ_X, NP, SPB><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
  } else {
    if (fp32) project_kernel<float, PJ_IN, NP, SPB><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
    else project_kernel<double, PJ_IN, NP, SPB><<<grid, 128, 0, st>>>(jt, b, x_in, c_out);
  }
}

cudaError_t launch_project(int mode, bool fp32, int nslots, int n_groups, int max_np, cudaStream_t st,
                           const JuncDev* jt, const BatchDev* b, const void* x_in, void* c_out,
                           bool one_slot_per_cta) {
  // slots per CTA: the projector values of an atom are loaded once for all of
  // them; a pool over several junctions takes one slot per CTA (atom g differs
  // between junctions)
  if (one_slot_per_cta && max_np <= 4) {
    launch_project_np<4, 1>(mode, fp32, dim3(n_groups, nslots), st, jt, b, x_in, c_out);
  } else if (one_slot_per_cta && max_np <= 9) {
    launch_project_np<9, 1>(mode, fp32, dim3(n_groups, nslots), st, jt, b, x_in, c_out);
  } else if (max_np <= 4) {
    launch_project_np<4, 4>(mode, fp32, dim3(n_groups, (nslots + 3) / 4), st, jt, b, x_in, c_out);
  } else if (max_np <= 9) {
    launch_project_np<9, 2>(mode, fp32, dim3(n_groups, (nslots + 1) / 2), st, jt, b, x_in, c_out);
  } else if (max_np <= kMaxGroupNp) {
    launch_project_np<kMaxGroupNp, 1>(mode, fp32, dim3(n_groups, nslots), st, jt, b, x_in, c_out);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_book(int nslots, int slot_it, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  book_kernel<<<(nslots + kBookWarps - 1) / kBookWarps, 32 * kBookWarps, 0, st>>>(jt, b, slot_it);
  return cudaGetLastError();
}

cudaError_t launch_sched(int nslots, int slot_it, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  (void)nslots;
  sched_kernel<<<1, kSchedThreads, 0, st>>>(jt, b, slot_it);
  return cudaGetLastError();
}

cudaError_t launch_x_update(bool fp32, int nslots, int nB, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  dim3 grid(nB, nslots);
  if (fp32) x_update_kernel<float><<<grid, kVecThreads, 0, st>>>(jt, b);
  else x_update_kernel<double><<<grid, kVecThreads, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_shift_init(int nT, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  const int bx = std::max(1, std::min(64, (nT + kVecThreads - 1) / kVecThreads));
  shift_init_kernel<<<dim3(bx, kListRows), kVecThreads, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_shift_update(int nslots, int nT, int n_shift, cudaStream_t st, const JuncDev* jt,
                                const BatchDev* b) {
  const int bx = std::max(1, (nT + kVecThreads - 1) / kVecThreads);
  shift_update_kernel<<<dim3(bx, nslots), kVecThreads, 3 * n_shift * sizeof(double2), st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_shift_emit(int nslots, int n_shift, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  shift_emit_kernel<<<dim3(n_shift, nslots), 256, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_tgoal(cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  tgoal_kernel<<<kListRows, 256, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_landauer(int n_e, const double* E, const double* T, int n_v, const double* V, double E_F,
                            double kT, double* I, cudaStream_t st) {
  landauer_kernel<<<n_v, 256, 0, st>>>(n_e, E, T, V, E_F, kT, I);
  return cudaGetLastError();
}

cudaError_t launch_list(cudaStream_t st, const BatchDev* b) {
  list_kernel<<<1, kSchedThreads, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_emit(int nslots, cudaStream_t st, const JuncDev* jt, const BatchDev* b) {
  emit_kernel<<<nslots, 256, 0, st>>>(jt, b);
  return cudaGetLastError();
}

cudaError_t launch_t_final(int n_e, int n_cols, cudaStream_t st, const double* t_all, const double* gr_cols,
                           double* T_out) {
  const int warps = 8;
  t_final_kernel<<<(n_e + warps - 1) / warps, 32 * warps, 0, st>>>(n_e, n_cols, t_all, gr_cols, T_out);
  return cudaGetLastError();
}

cudaError_t launch_grad_sys(int nsys, long long N, cudaStream_t st, const double2* lam, const double2* x,
                            const double* wt, double* g) {
  grad_sys_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(nsys, N, lam, x, wt, g);
  return cudaGetLastError();
}

}  // namespace rsn
