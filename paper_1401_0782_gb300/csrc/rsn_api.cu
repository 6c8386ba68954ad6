// C-ABI entry points, device-side setup of the operator data, and the host
// driver of the streaming COCG solver with FP64 reliable updates.
//
// Systems A(E_k) x_k = b_k wait in a queue; a fixed pool of S slots holds the
// ones being solved.  One iteration of the solver is a fixed sequence of
// kernels (see vec_kernels.cu): new systems are initialised, systems whose
// recurrence reached its target get an FP64 true residual (which either
// finishes them or replaces the recurrence residual, keeping the search
// direction), finished slots take the next queued systems, and every active
// slot does one COCG iteration.  `graph_iters` iterations are captured once as
// a CUDA graph and replayed; between replays the host reads a few integers
// (queue position, busy slots).  Everything else stays on the GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rsnegf.h"
#include "rsn_internal.h"

using namespace rsn;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    release();
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = bytes;
    return cudaSuccess;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct Tiling {
  int TY = 0, Lz = 0, ytiles = 0, ztiles = 0, n = 0, ppt = 1, threads = 32;
  size_t smem = 0;
  bool tma = false;   // whole-plane tile streamed by bulk copies (op_kernel_tma)
  bool pair = false;  // FP32 point-pair kernel with plane streaming (op_pair_kernel)
  bool plane = false; // FP32 one-point-per-thread kernel with plane streaming (op_plane_kernel)
  bool big = false;   // its one-CTA-per-SM variant (planes of more than 2 * kPairThreads points)
};

// Slot pool of the streaming solver (sized for S slots of N points).
struct Workspace {
  int slots = 0;
  bool fp32 = false;
  long long N = 0;
  int PA = 0, PB = 0, n_proj = 0;
  DevBuf Xslot, r, p0, p1, q, d;
  DevBuf state, sys, junc, E, col, voff, xo, xfo, iters, total_iters, cyc_iters, n_upd, restart, stall, warm, rho_cur, beta_cur;
  DevBuf bnorm2, sigma, rlast2, rrec2, tol2;
  DevBuf rho0, nrm0, t0, tlast, gcnt, gphase, tgoal, rgoal, rho, nrm, mu, c_r, c_p, c_x, sched, counters, lst, lst_n,
      inlist, fslot, c_e;
  int generation = 0;
};

// Per-call system queue and outputs.
struct CallBufs {
  DevBuf sys_junc, sys_E, sys_col, sys_xo, sys_xfo, sys_dep, sys_bn2, sys_started, out_iters, out_relres, out_status,
      out_t;
  DevBuf X0, X1, wt, g, t_all, gr_cols, Td;
  // shifted systems
  DevBuf sh_sig, sh_idx, sh_xs, sh_ps, sh_pi, sh_cit, sh_alpha, sh_beta, sh_rn2, sh_ts, sh_sit, sh_srel;
  // Landauer current
  DevBuf lE, lT, lV, lI;
};

// Shifted-system part of a stream (rsn_*_shifted): the energies' shifts from
// the seed, the tracked points and where the shifted iterates go.
struct ShiftSpec {
  int n_shift = 0;
  std::vector<double> sig;  // E_e - E_seed
  int nT = 0;
  const int* idx = nullptr;  // device: tracked grid points
  double2* xs_out = nullptr; // caller's [n_e][n_cols][N] output (every point tracked), or null: slot storage
  long long n_cols = 0;
};

// A slot pool over several junctions of one device (rsn_batch_transmission):
// the per-junction operator data stay with their contexts; one JuncDev per
// junction carries its tilings, and each slot works on its system's junction.
struct PoolSpec {
  int K = 0, R = 0;
  long long N = 0;  // the largest junction: slot vectors are this long
  int n_proj = 0, n_groups = 0, max_np = 1, nB = 0, nS = 0, PA = 0, PB = 0;
  Tiling inner[4];                        // launch configuration per operator kind (OpKind)
  bool has[4] = {false, false, false, false};
  Tiling resid;                           // launch configuration of the true-residual kernel
  const JuncDev* ji = nullptr;            // device: K JuncDev with the COCG tilings
  const JuncDev* jr = nullptr;            // device: K JuncDev with the residual tilings
};

// Buffers of the block COCG solver (rsn_*_block): FP32 block vectors W, P, AP,
// D and the FP64 iterate / residual of every member of a wave of blocks, the
// b x b state of each block, and the apply lists of the active members.
struct BlkBufs {
  DevBuf W, P, AP, D, X, R, part, xi, QQ, xi0n, alpha, axi, tinv, tinv64, beta, flag, its, rpart, rn, tt, blist, col;
  DevBuf vE, vjunc, voff, cbuf, dev, bdev, jd, t_all, gr_cols, Td, stat, icap;
};

struct GraphKey {
  int fp32, slots, iters, generation, proj, timing, n_shift, nT;
  bool operator<(const GraphKey& o) const {
    return std::tie(fp32, slots, iters, generation, proj, timing, n_shift, nT) <
           std::tie(o.fp32, o.slots, o.iters, o.generation, o.proj, o.timing, o.n_shift, o.nT);
  }
};

}  // namespace

struct rsn_ctx {
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t st = nullptr;
  cudaStream_t st2 = nullptr;  // second stream: the true-residual path beside the COCG step
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr, ev_fork = nullptr, ev_join = nullptr;
  std::string err;

  bool has_grid = false, has_v = false, has_cap = false;
  int nx = 0, ny = 0, nz = 0, R = 0;
  double h = 0;
  long long N = 0;
  std::vector<double> v, gl, gr;
  int n_proj = 0;
  std::vector<int64_t> poff;
  std::vector<int32_t> pidx;
  std::vector<double> pval, pekb;
  bool dirty = true;

  // device operator data
  DevBuf dg64, dg32, gld, L_idx, L_gam, inv_ptr, inv_p0, inv_q64, inv_q32, sup_pts;
  int n_sup = 0;
  DevBuf grp_ptr, grp_p0, grp_np, grp_voff, grp_idx, grp_val64, grp_val32, ekb;
  int n_groups = 0, nL = 0, max_np = 1;
  JuncDev jh{};
  DevBuf jd;  // device JuncDev (one per launch configuration, uploaded before a batch)
  DevBuf pool_jd;  // device JuncDev of a slot pool over several junctions (this context owns the pool)

  Workspace ws;
  CallBufs cb;
  BlkBufs bb;
  DevBuf bd;  // device BatchDev: [0] streaming solver, [1] rsn_apply
  std::map<GraphKey, cudaGraphExec_t> graphs;
  int* sched_host = nullptr;  // pinned mirror of BatchDev::sched
  unsigned long long* cnt_host = nullptr;  // pinned mirror of BatchDev::counters

  // stats of the last solve
  int64_t st_iters = 0, st_sweeps = 0, st_launches = 0, st_fallback = 0;
  double st_ms = 0.0;
  // live kernel timing (opts.timing): [0] COCG operator kernel, [1] COCG update kernel
  std::vector<cudaEvent_t> tev;  // 4 per graph iteration
  int64_t ks_launches[2] = {0, 0};
  double ks_ms[2] = {0, 0}, ks_bytes[2] = {0, 0};
  int tile_override[4] = {0, 0, 0, 0};  // TY, Lz, ppt, -1 = plane-streaming (TMA) kernel
};

static std::string g_create_err;

#define RSN_FAIL(ctx, code, ...)                                   \
  do {                                                             \
    char _b[512];                                                  \
    snprintf(_b, sizeof(_b), __VA_ARGS__);                         \
    (ctx)->err = _b;                                               \
    return code;                                                   \
  } while (0)
#define RSN_CUDA(ctx, call)                                                               \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) {                                                              \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(_e);                    \
      return _e == cudaErrorMemoryAllocation ? RSN_ENOMEM : RSN_ECUDA;                    \
    }                                                                                     \
  } while (0)

// ---------------------------------------------------------------------------
// finite-difference weights: c_k = 2(-1)^{k+1}(R!)^2 / (k^2 (R-k)! (R+k)!),
// c_0 = -2 sum_k c_k (central second derivative of order 2R, h = 1)
// ---------------------------------------------------------------------------
static void fd_weights(int R, double* c) {
  auto fact = [](int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  double s = 0.0;
  for (int k = 1; k <= R; ++k) {
    c[k] = 2.0 * ((k & 1) ? 1.0 : -1.0) * fact(R) * fact(R) / ((double)k * k * fact(R - k) * fact(R + k));
    s += c[k];
  }
  c[0] = -2.0 * s;
}

static void clear_graphs(rsn_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// ---------------------------------------------------------------------------
// tiling of the operator kernel
// ---------------------------------------------------------------------------
// Tiling overrides (rsn_set_tiling): TY rows, Lz planes, ppt points per
// thread; ppt = -1 selects the whole-plane bulk-copy kernel of one point per
// thread with a register-shifted queue, ppt = -2 the FP32 point-pair kernel,
// ppt = -3 the FP32 plane kernel (one point per thread, unrolled ring);
// automatic: the point-pair kernel where it applies (nx even), else the plane
// kernel, else the register kernel.
// `streamable`: the vectors of this launch are 16-byte aligned (bulk copies).
static Tiling choose_tiling(const rsn_ctx* c, bool compute64, int mode, int nslots, bool streamable = true) {
  Tiling t;
  const int nx = c->nx, ny = c->ny, nz = c->nz, R = c->R;
  const long long pl = (long long)nx * ny;
  // FP32 point-pair kernel: whole planes, nx even (16-byte pairs), at most
  // 2 * kPairThreadsBig points per plane, no explicit register tile requested
  const bool reg_forced = c->tile_override[0] > 0 || c->tile_override[2] > 0 || c->tile_override[3] == -1;
  auto z_chunks = [&](int per_sm) {
    int zt = (4 * per_sm * 152 + nslots - 1) / nslots;
    zt = std::max(1, std::min(zt, std::max(1, nz / (2 * R + 2))));
    if (c->tile_override[1] > 0) zt = (nz + c->tile_override[1] - 1) / c->tile_override[1];
    t.Lz = (nz + zt - 1) / zt;
    t.ztiles = (nz + t.Lz - 1) / t.Lz;
    t.n = t.ztiles;
    t.TY = ny;
    t.ytiles = 1;
  };
  if (!compute64 && mode != OP_RESID && streamable && !reg_forced && c->tile_override[3] != -3 && nx % 2 == 0) {
    const int thr = (int)(((pl / 2) + 31) / 32 * 32);
    const size_t sm = op_pair_smem_bytes(mode, R, nx, ny, c->n_proj);
    if (thr <= kPairThreadsBig && sm <= 200 * 1024) {
      t.pair = true;
      t.big = thr > kPairThreads;
      t.threads = thr;
      t.smem = sm;
      t.ppt = 2;
      z_chunks(t.big ? 1 : 2);
      return t;
    }
  }
  if (!compute64 && mode != OP_RESID && streamable && !reg_forced && c->tile_override[3] != -2 && pl % 2 == 0 &&
      pl <= kPlaneThreads) {
    const size_t sm = op_pair_smem_bytes(mode, R, nx, ny, c->n_proj);
    if (sm <= 100 * 1024) {
      t.plane = true;
      t.threads = (int)((pl + 31) / 32 * 32);
      t.smem = sm;
      t.ppt = 1;
      z_chunks(2);
      return t;
    }
  }
  // register-prefetch kernel: one point per thread by default (64 registers,
  // 4 CTAs per SM), as many whole x rows per tile as fit 256 threads; the
  // autotuner may choose otherwise
  int TY = std::max(1, std::min(ny, 256 / std::max(1, nx)));
  {
    const int yt = (ny + TY - 1) / TY;
    TY = (ny + yt - 1) / yt;
  }
  int ppt = 1;
  if (c->tile_override[0] > 0) TY = std::min(ny, c->tile_override[0]);
  if (c->tile_override[2] > 0) ppt = std::min(4, c->tile_override[2]);
  int threads = (nx * TY + ppt - 1) / ppt;
  threads = ((threads + 31) / 32) * 32;
  while (threads > 256 && ppt < 4) {
    ++ppt;
    threads = (((nx * TY + ppt - 1) / ppt) + 31) / 32 * 32;
  }
  while (threads > 256 && TY > 1) {  // still too many: split the plane into more y tiles
    TY = (TY + 1) / 2;
    threads = (((nx * TY + ppt - 1) / ppt) + 31) / 32 * 32;
  }
  t.TY = TY;
  t.ytiles = (ny + TY - 1) / TY;
  t.ppt = ppt;
  t.threads = threads;
  int want = 8 * 152;
  int zt = (want + nslots * t.ytiles - 1) / (nslots * t.ytiles);
  zt = std::max(1, std::min(zt, std::max(1, nz / (2 * R + 2))));
  if (c->tile_override[1] > 0) zt = (nz + c->tile_override[1] - 1) / c->tile_override[1];
  // few systems need a true residual at a time and it sits on every
  // iteration's critical path: two planes per CTA whatever the operator
  // tiling, so that each CTA marches through 2R + 2 planes only (latency, not
  // bandwidth, bounds it)
  if (mode == OP_RESID) zt = std::max(1, nz / 2);
  t.Lz = (nz + zt - 1) / zt;
  t.ztiles = (nz + t.Lz - 1) / t.Lz;
  t.n = t.ytiles * t.ztiles;
  t.smem = op_smem_bytes(!compute64, mode, R, TY, nx, c->n_proj);
  // whole-plane bulk-copy kernel (on request): FP32 COCG / apply on planes
  // whose byte sizes keep every bulk copy 16-byte aligned
  if (!compute64 && mode != OP_RESID && streamable && pl <= 1024 && (pl * 8) % 16 == 0 && (c->N * 8) % 16 == 0 &&
      c->tile_override[3] == -1) {
    const size_t sm = op_tma_smem_bytes(true, mode, R, nx, ny, c->n_proj);
    if (sm <= 200 * 1024) {
      t.TY = ny;
      t.ytiles = 1;
      t.n = t.ztiles;
      t.tma = true;
      t.smem = sm;
      t.threads = (int)((pl + 31) / 32 * 32);
    }
  }
  return t;
}

// Operator launch (COCG or apply) with a tiling from choose_tiling; the
// JuncDev copy `jt` must carry the same tiling.
static cudaError_t launch_inner(const rsn_ctx* c, const Tiling& t, int mode, bool fp32, int nslots, cudaStream_t st,
                                const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out,
                                const void* c_in) {
  const dim3 grid(t.n, nslots);
  if (t.plane) return launch_op_plane(mode, c->R, grid, t.threads, t.smem, st, jt, b, x_in, y_out, c_in);
  if (t.pair) return launch_op_pair(mode, c->R, t.big, grid, t.threads, t.smem, st, jt, b, x_in, y_out, c_in);
  if (t.tma) return launch_op_tma(mode, fp32, c->R, grid, t.threads, t.smem, st, jt, b, x_in, y_out, c_in);
  return launch_op(mode, fp32, c->R, t.ppt, grid, t.threads, t.smem, st, jt, b, x_in, y_out, c_in);
}

// ---------------------------------------------------------------------------
// upload of the operator data (done lazily before the first solve/apply)
// ---------------------------------------------------------------------------
static rsn_status commit_setup(rsn_ctx* c) {
  if (!c->has_grid) RSN_FAIL(c, RSN_ESTATE, "rsn_set_grid has not been called");
  if (!c->has_v) RSN_FAIL(c, RSN_ESTATE, "rsn_set_potential has not been called");
  if (!c->has_cap) RSN_FAIL(c, RSN_ESTATE, "rsn_set_cap has not been called");
  if (!c->dirty) return RSN_OK;
  const long long N = c->N;
  double cw[kMaxR + 1] = {0};
  fd_weights(c->R, cw);
  const double ih2 = 1.0 / (2.0 * c->h * c->h);
  std::vector<double2> dg(N);
  std::vector<float2> dgf(N);
  for (long long i = 0; i < N; ++i) {
    dg[i] = make_double2(-c->v[i] + 3.0 * cw[0] * ih2, c->gl[i] + c->gr[i]);
    // FP32 kernels use the difference form of the stencil: no FD diagonal here
    dgf[i] = make_float2((float)(-c->v[i]), (float)dg[i].y);
  }
  RSN_CUDA(c, c->dg64.ensure(N * sizeof(double2)));
  RSN_CUDA(c, c->dg32.ensure(N * sizeof(float2)));
  RSN_CUDA(c, c->gld.ensure(N * sizeof(double)));
  RSN_CUDA(c, cudaMemcpy(c->dg64.p, dg.data(), N * sizeof(double2), cudaMemcpyHostToDevice));
  RSN_CUDA(c, cudaMemcpy(c->dg32.p, dgf.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
  RSN_CUDA(c, cudaMemcpy(c->gld.p, c->gl.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  std::vector<int> lidx;
  std::vector<double> lgam;
  for (long long i = 0; i < N; ++i)
    if (c->gl[i] > 0.0) {
      lidx.push_back((int)i);
      lgam.push_back(c->gl[i]);
    }
  c->nL = (int)lidx.size();
  RSN_CUDA(c, c->L_idx.ensure(std::max<size_t>(1, lidx.size()) * sizeof(int)));
  RSN_CUDA(c, c->L_gam.ensure(std::max<size_t>(1, lgam.size()) * sizeof(double)));
  if (!lidx.empty()) {
    RSN_CUDA(c, cudaMemcpy(c->L_idx.p, lidx.data(), lidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    RSN_CUDA(c, cudaMemcpy(c->L_gam.p, lgam.data(), lgam.size() * sizeof(double), cudaMemcpyHostToDevice));
  }

  // projectors: atoms = runs of consecutive projectors with identical supports
  const int np = c->n_proj;
  std::vector<int> gptr{0}, gp0, gnp, gidx;
  std::vector<long long> gvoff;
  std::vector<double> gval;
  std::vector<int> cnt(N + 1, 0);
  if (np > 0) {
    int p = 0;
    while (p < np) {
      const int64_t a0 = c->poff[p], a1 = c->poff[p + 1];
      int q = p + 1;
      while (q < np && q - p < kMaxGroupNp && c->poff[q + 1] - c->poff[q] == a1 - a0 &&
             std::equal(c->pidx.begin() + c->poff[q], c->pidx.begin() + c->poff[q + 1], c->pidx.begin() + a0))
        ++q;
      const int len = (int)(a1 - a0);
      gp0.push_back(p);
      gnp.push_back(q - p);
      gvoff.push_back((long long)gval.size());
      for (int k = p; k < q; ++k)
        for (int e = 0; e < len; ++e) gval.push_back(c->pval[c->poff[k] + e]);
      for (int e = 0; e < len; ++e) gidx.push_back(c->pidx[a0 + e]);
      gptr.push_back((int)gidx.size());
      p = q;
    }
  }
  c->n_groups = (int)gp0.size();
  c->max_np = 1;
  for (int v : gnp) c->max_np = std::max(c->max_np, v);
  // per grid point, one entry per atom whose support holds it: the atom's
  // first projector and its projector values there, padded with zeros to
  // quads (4 values) so that the operator kernel reads them as vectors
  const int nq = (c->max_np + 3) / 4;
  const int G = c->n_groups;
  for (int g = 0; g < G; ++g)
    for (int k = gptr[g]; k < gptr[g + 1]; ++k) cnt[gidx[k] + 1]++;
  std::vector<int> sup;  // grid points inside at least one projector support
  for (long long i = 0; i < N; ++i) {
    if (cnt[i + 1] > 0) sup.push_back((int)i);
    cnt[i + 1] += cnt[i];
  }
  c->n_sup = (int)sup.size();
  const size_t nent = (size_t)cnt[N];
  std::vector<int> ip0(std::max<size_t>(1, nent)), fill(cnt.begin(), cnt.end() - 1);
  std::vector<double> iq64(std::max<size_t>(1, nent) * 4 * nq, 0.0);
  for (int g = 0; g < G; ++g) {
    const int len = gptr[g + 1] - gptr[g];
    for (int k = 0; k < len; ++k) {
      const int i = gidx[gptr[g] + k];
      const int e = fill[i]++;
      ip0[e] = gp0[g];
      for (int j = 0; j < gnp[g]; ++j) iq64[(size_t)e * 4 * nq + j] = gval[gvoff[g] + (size_t)j * len + k];
    }
  }
  std::vector<float> iq32(iq64.begin(), iq64.end()), gvalf(gval.begin(), gval.end());
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = b.ensure(std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    if (bytes) return cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice);
    return cudaSuccess;
  };
  RSN_CUDA(c, up(c->inv_ptr, cnt.data(), (N + 1) * sizeof(int)));
  RSN_CUDA(c, up(c->inv_p0, ip0.data(), nent * sizeof(int)));
  RSN_CUDA(c, up(c->sup_pts, sup.data(), sup.size() * sizeof(int)));
  RSN_CUDA(c, up(c->inv_q64, iq64.data(), nent * 4 * nq * sizeof(double)));
  RSN_CUDA(c, up(c->inv_q32, iq32.data(), nent * 4 * nq * sizeof(float)));
  RSN_CUDA(c, up(c->grp_ptr, gptr.data(), gptr.size() * sizeof(int)));
  RSN_CUDA(c, up(c->grp_p0, gp0.data(), gp0.size() * sizeof(int)));
  RSN_CUDA(c, up(c->grp_np, gnp.data(), gnp.size() * sizeof(int)));
  RSN_CUDA(c, up(c->grp_voff, gvoff.data(), gvoff.size() * sizeof(long long)));
  RSN_CUDA(c, up(c->grp_idx, gidx.data(), gidx.size() * sizeof(int)));
  RSN_CUDA(c, up(c->grp_val64, gval.data(), gval.size() * sizeof(double)));
  RSN_CUDA(c, up(c->grp_val32, gvalf.data(), gvalf.size() * sizeof(float)));
  RSN_CUDA(c, up(c->ekb, c->pekb.data(), c->pekb.size() * sizeof(double)));

  JuncDev& J = c->jh;
  memset(&J, 0, sizeof(J));
  J.nx = c->nx;
  J.ny = c->ny;
  J.nz = c->nz;
  J.plane = c->nx * c->ny;
  J.N = N;
  for (int m = 1; m <= c->R; ++m) {
    J.w64[m] = cw[m] * ih2;
    J.w32[m] = (float)(cw[m] * ih2);
  }
  J.nB = (int)((N + kVecPts - 1) / kVecPts);
  J.dg64 = c->dg64.as<double2>();
  J.dg32 = c->dg32.as<float2>();
  J.gl = c->gld.as<double>();
  J.nL = c->nL;
  J.L_idx = c->L_idx.as<int>();
  J.L_gam = c->L_gam.as<double>();
  J.n_proj = np;
  J.n_groups = c->n_groups;
  J.inv_ptr = c->inv_ptr.as<int>();
  J.inv_nq = (c->max_np + 3) / 4;
  J.inv_p0 = c->inv_p0.as<int>();
  J.inv_q64 = c->inv_q64.as<double2>();
  J.inv_q32 = c->inv_q32.as<float4>();
  J.sup_pts = c->sup_pts.as<int>();
  J.n_sup = c->n_sup;
  J.nS = (c->n_sup + kVecPts - 1) / kVecPts;
  J.grp_ptr = c->grp_ptr.as<int>();
  J.grp_p0 = c->grp_p0.as<int>();
  J.grp_np = c->grp_np.as<int>();
  J.grp_voff = c->grp_voff.as<long long>();
  J.grp_idx = c->grp_idx.as<int>();
  J.grp_val64 = c->grp_val64.as<double>();
  J.grp_val32 = c->grp_val32.as<float>();
  J.ekb = c->ekb.as<double>();
  RSN_CUDA(c, c->jd.ensure(4 * sizeof(JuncDev)));
  c->dirty = false;
  clear_graphs(c);
  c->ws.generation++;
  return RSN_OK;
}

// Device JuncDev copies for one launch configuration: copy 0 carries the tiling
// of the COCG / apply operator kernel, copy 1 that of the FP64 true-residual
// kernel; both record the residual kernel's CTA count (nR) for its partials.
struct LaunchCfg {
  Tiling inner, resid;
  const JuncDev* jt_inner;  // device pointer: tiling of the COCG / apply kernel
  const JuncDev* jt_resid;  // device pointer: tiling of the residual kernel
};

static rsn_status make_cfg(rsn_ctx* c, const Tiling& inner, const Tiling& resid, LaunchCfg& cfg) {
  cfg.inner = inner;
  cfg.resid = resid;
  JuncDev js[2] = {c->jh, c->jh};
  for (int k = 0; k < 2; ++k) {
    const Tiling& t = k == 0 ? cfg.inner : cfg.resid;
    js[k].TY = t.TY;
    js[k].Lz = t.Lz;
    js[k].ytiles = t.ytiles;
    js[k].ztiles = t.ztiles;
    js[k].nA = t.n;
    js[k].nR = cfg.resid.n;
    js[k].kind = k == 1 ? kOpReg : t.plane ? kOpPlane : t.pair ? kOpPair : t.tma ? kOpTma : kOpReg;
  }
  RSN_CUDA(c, cudaMemcpyAsync(c->jd.p, js, 2 * sizeof(JuncDev), cudaMemcpyHostToDevice, c->st));
  cfg.jt_inner = c->jd.as<JuncDev>();
  cfg.jt_resid = c->jd.as<JuncDev>() + 1;
  return RSN_OK;
}

// the solver's tilings: COCG operator in the inner precision, FP64 true residual
static rsn_status make_cfg(rsn_ctx* c, bool fp32, int nslots, LaunchCfg& cfg) {
  return make_cfg(c, choose_tiling(c, !fp32, OP_COCG, nslots), choose_tiling(c, true, OP_RESID, nslots), cfg);
}

extern "C" {

void rsn_default_opts(int precision, rsn_solver_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = precision == RSN_MIXED ? RSN_MIXED : RSN_FP64;
  if (o->precision == RSN_MIXED) {
    o->tol = 1e-10;
    o->tol_inner = 1e-1;
    o->max_iter = 3000;  // slower systems are handed to the FP64 fallback
    o->tol_T = 1e-7;
  } else {
    o->tol = 1e-13;
    o->tol_inner = 1e-6;
    o->max_iter = 20000;
    o->tol_T = 3e-11;
  }
  o->tol_adjoint = 0.0;  // the adjoint systems take tol
  o->max_outer = 64;
  o->deadline_ms = 0.0;
  o->rhs_block = 0;
  o->use_graph = 1;
  o->graph_iters = 16;
  o->timing = 0;
}

rsn_status rsn_create(rsn_ctx** out, int device, void* cuda_stream) {
  if (!out) {
    g_create_err = "rsn_create: out is NULL";
    return RSN_EINVAL;
  }
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    g_create_err = std::string("rsn_create: no CUDA device ") + std::to_string(device) + " (" +
                   (e != cudaSuccess ? cudaGetErrorString(e) : "out of range") + ")";
    return e != cudaSuccess ? RSN_ECUDA : RSN_EINVAL;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    g_create_err = std::string("rsn_create: cudaSetDevice: ") + cudaGetErrorString(e);
    return RSN_ECUDA;
  }
  rsn_ctx* c = new rsn_ctx();
  c->device = device;
  c->user_stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&c->t0) != cudaSuccess || cudaEventCreate(&c->t1) != cudaSuccess ||
      cudaMallocHost(&c->sched_host, (3 + 2 * kMaxGraphIters) * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->cnt_host, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    g_create_err = "rsn_create: stream/event/pinned allocation failed";
    rsn_destroy(c);
    return RSN_ECUDA;
  }
  *out = c;
  g_create_err.clear();
  return RSN_OK;
}

rsn_status rsn_destroy(rsn_ctx* c) {
  if (!c) return RSN_OK;
  cudaSetDevice(c->device);
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->st2) cudaStreamSynchronize(c->st2);
  clear_graphs(c);
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  if (c->sched_host) cudaFreeHost(c->sched_host);
  if (c->cnt_host) cudaFreeHost(c->cnt_host);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->t0) cudaEventDestroy(c->t0);
  if (c->t1) cudaEventDestroy(c->t1);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
  return RSN_OK;
}

rsn_status rsn_set_grid(rsn_ctx* c, int nx, int ny, int nz, double h, int R) {
  if (!c) return RSN_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1) RSN_FAIL(c, RSN_EINVAL, "grid sizes must be >= 1");
  if ((long long)nx * ny > kMaxPlane) RSN_FAIL(c, RSN_EINVAL, "nx*ny = %lld exceeds %d", (long long)nx * ny, kMaxPlane);
  if (!(h > 0) || !std::isfinite(h)) RSN_FAIL(c, RSN_EINVAL, "h must be positive");
  if (R < 1 || R > kMaxR) RSN_FAIL(c, RSN_EINVAL, "fd_half_order must be in 1..%d", kMaxR);
  const long long N = (long long)nx * ny * nz;
  if (N >= (1LL << 31)) RSN_FAIL(c, RSN_EINVAL, "grid too large");
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->h = h;
  c->R = R;
  c->N = N;
  c->has_grid = true;
  c->has_v = c->has_cap = false;
  c->n_proj = 0;
  c->poff.assign(1, 0);
  c->pidx.clear();
  c->pval.clear();
  c->pekb.clear();
  c->dirty = true;
  c->err.clear();
  return RSN_OK;
}

rsn_status rsn_set_potential(rsn_ctx* c, const double* v) {
  if (!c) return RSN_EINVAL;
  if (!c->has_grid) RSN_FAIL(c, RSN_ESTATE, "rsn_set_grid has not been called");
  if (!v) RSN_FAIL(c, RSN_EINVAL, "v_loc is NULL");
  for (long long i = 0; i < c->N; ++i)
    if (!std::isfinite(v[i])) RSN_FAIL(c, RSN_EINVAL, "v_loc[%lld] is not finite", i);
  c->v.assign(v, v + c->N);
  c->has_v = true;
  c->dirty = true;
  return RSN_OK;
}

rsn_status rsn_set_cap(rsn_ctx* c, const double* gl, const double* gr) {
  if (!c) return RSN_EINVAL;
  if (!c->has_grid) RSN_FAIL(c, RSN_ESTATE, "rsn_set_grid has not been called");
  if (!gl || !gr) RSN_FAIL(c, RSN_EINVAL, "gamma_l / gamma_r is NULL");
  for (long long i = 0; i < c->N; ++i)
    if (!(gl[i] >= 0.0) || !(gr[i] >= 0.0) || !std::isfinite(gl[i]) || !std::isfinite(gr[i]))
      RSN_FAIL(c, RSN_EINVAL, "absorbing potentials must be finite and >= 0 (index %lld)", i);
  c->gl.assign(gl, gl + c->N);
  c->gr.assign(gr, gr + c->N);
  c->has_cap = true;
  c->dirty = true;
  return RSN_OK;
}

rsn_status rsn_set_projectors(rsn_ctx* c, int n_proj, const int64_t* off, const int32_t* idx, const double* val,
                              const double* ekb) {
  if (!c) return RSN_EINVAL;
  if (!c->has_grid) RSN_FAIL(c, RSN_ESTATE, "rsn_set_grid has not been called");
  if (n_proj < 0 || n_proj > 65536) RSN_FAIL(c, RSN_EINVAL, "n_proj out of range");
  if (n_proj == 0) {
    c->n_proj = 0;
    c->poff.assign(1, 0);
    c->pidx.clear();
    c->pval.clear();
    c->pekb.clear();
    c->dirty = true;
    return RSN_OK;
  }
  if (!off || !idx || !val || !ekb) RSN_FAIL(c, RSN_EINVAL, "projector arrays must not be NULL");
  if (off[0] != 0) RSN_FAIL(c, RSN_EINVAL, "offsets[0] must be 0");
  for (int p = 0; p < n_proj; ++p) {
    if (off[p + 1] < off[p]) RSN_FAIL(c, RSN_EINVAL, "offsets must be non-decreasing (p = %d)", p);
    if (!std::isfinite(ekb[p])) RSN_FAIL(c, RSN_EINVAL, "e_kb[%d] is not finite", p);
  }
  const int64_t nnz = off[n_proj];
  if (nnz >= (1LL << 31)) RSN_FAIL(c, RSN_EINVAL, "too many projector entries");
  for (int64_t e = 0; e < nnz; ++e) {
    if (idx[e] < 0 || idx[e] >= c->N) RSN_FAIL(c, RSN_EINVAL, "projector index %d out of range", idx[e]);
    if (!std::isfinite(val[e])) RSN_FAIL(c, RSN_EINVAL, "projector value %lld is not finite", (long long)e);
  }
  c->n_proj = n_proj;
  c->poff.assign(off, off + n_proj + 1);
  c->pidx.assign(idx, idx + nnz);
  c->pval.assign(val, val + nnz);
  c->pekb.assign(ekb, ekb + n_proj);
  c->dirty = true;
  return RSN_OK;
}

const char* rsn_last_error(const rsn_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

rsn_status rsn_kernel_stats(const rsn_ctx* c, int kind, int64_t* launches, double* ms, double* bytes) {
  if (!c || kind < 0 || kind > 1) return RSN_EINVAL;
  if (launches) *launches = c->ks_launches[kind];
  if (ms) *ms = c->ks_ms[kind];
  if (bytes) *bytes = c->ks_bytes[kind];
  return RSN_OK;
}

rsn_status rsn_last_stats(const rsn_ctx* c, int64_t* it, int64_t* sw, int64_t* la, double* ms, int64_t* fb) {
  if (!c) return RSN_EINVAL;
  if (fb) *fb = c->st_fallback;
  if (it) *it = c->st_iters;
  if (sw) *sw = c->st_sweeps;
  if (la) *la = c->st_launches;
  if (ms) *ms = c->st_ms;
  return RSN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// stream ordering with the caller's stream
// ---------------------------------------------------------------------------
static rsn_status enter(rsn_ctx* c) {
  RSN_CUDA(c, cudaSetDevice(c->device));
  RSN_CUDA(c, cudaEventRecord(c->ev_in, c->user_stream));
  RSN_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_in, 0));
  return RSN_OK;
}
static rsn_status leave(rsn_ctx* c) {
  RSN_CUDA(c, cudaEventRecord(c->ev_out, c->st));
  RSN_CUDA(c, cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
  return RSN_OK;
}

// ---------------------------------------------------------------------------
// slot pool
// ---------------------------------------------------------------------------
static size_t slot_bytes(const rsn_ctx* c, bool fp32) {
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  return (size_t)c->N * (sizeof(double2) + 5 * el) + 8192;
}

// Slots: enough systems in flight to fill the GPU, few enough (relative to the
// queue) that the drain at the end of the queue stays short, and within memory.
static int choose_slots(rsn_ctx* c, const rsn_solver_opts* o, long long nsys, size_t reserved,
                        size_t extra_per_slot = 0, long long N_pool = 0) {
  if (o->rhs_block > 0) return (int)std::max<long long>(1, std::min<long long>(o->rhs_block, nsys));
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const double avail = fr > reserved ? 0.6 * (double)(fr - reserved) : 0.0;
  const size_t per_slot = N_pool > 0 ? slot_bytes(c, o->precision == RSN_MIXED) * (size_t)N_pool / (size_t)c->N
                                     : slot_bytes(c, o->precision == RSN_MIXED);
  long long cap = (long long)(avail / (double)(per_slot + extra_per_slot));
  cap = std::max<long long>(1, std::min<long long>(cap, 8192));
  // one slot per system up to 2048: a stream then ends with its slowest
  // system instead of with a second wave of systems that waited for slots
  const long long want = std::min<long long>(nsys, 2048);
  return (int)std::max<long long>(1, std::min(want, cap));
}

static rsn_status ensure_ws(rsn_ctx* c, bool fp32, int S, const PoolSpec* pool = nullptr) {
  Workspace& w = c->ws;
  const long long N = pool ? pool->N : c->N;
  const int n_proj = pool ? pool->n_proj : c->n_proj;
  int PA, PB;
  if (pool) {
    PA = pool->PA;
    PB = pool->PB;
  } else {
    const Tiling ti = choose_tiling(c, !fp32, OP_COCG, S), tr = choose_tiling(c, true, OP_RESID, S);
    // mu partials: the operator tiles', then one per atom (projection kernel)
    PA = std::max(ti.n + c->n_groups, tr.n);
    PB = c->jh.nB;
  }
  if (w.slots == S && w.fp32 == fp32 && w.N == N && w.PA == PA && w.PB == PB && w.n_proj == n_proj)
    return RSN_OK;
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  const size_t vb = (size_t)S * N;
  RSN_CUDA(c, w.Xslot.ensure(vb * sizeof(double2)));
  RSN_CUDA(c, w.r.ensure(vb * el));
  RSN_CUDA(c, w.p0.ensure(vb * el));
  RSN_CUDA(c, w.p1.ensure(vb * el));
  RSN_CUDA(c, w.q.ensure(vb * el));
  RSN_CUDA(c, w.d.ensure(vb * el));
  const size_t si = S * sizeof(int), sd = S * sizeof(double), sl = S * sizeof(long long);
  RSN_CUDA(c, w.state.ensure(si));
  RSN_CUDA(c, w.sys.ensure(si));
  RSN_CUDA(c, w.junc.ensure(si));
  RSN_CUDA(c, w.E.ensure(sd));
  RSN_CUDA(c, w.col.ensure(si));
  RSN_CUDA(c, w.voff.ensure(sl));
  RSN_CUDA(c, w.xo.ensure(sl));
  RSN_CUDA(c, w.xfo.ensure(sl));
  RSN_CUDA(c, w.iters.ensure(si));
  RSN_CUDA(c, w.total_iters.ensure(si));
  RSN_CUDA(c, w.cyc_iters.ensure(si));
  RSN_CUDA(c, w.n_upd.ensure(si));
  RSN_CUDA(c, w.restart.ensure(si));
  RSN_CUDA(c, w.stall.ensure(si));
  RSN_CUDA(c, w.warm.ensure(si));
  RSN_CUDA(c, w.rho_cur.ensure(S * sizeof(double2)));
  RSN_CUDA(c, w.beta_cur.ensure(S * sizeof(double2)));
  RSN_CUDA(c, w.bnorm2.ensure(sd));
  RSN_CUDA(c, w.sigma.ensure(sd));
  RSN_CUDA(c, w.rlast2.ensure(sd));
  RSN_CUDA(c, w.rrec2.ensure(sd));
  RSN_CUDA(c, w.tol2.ensure(sd));
  RSN_CUDA(c, w.rho0.ensure((size_t)S * PA * sizeof(double2)));
  RSN_CUDA(c, w.nrm0.ensure((size_t)S * PA * sizeof(double)));
  RSN_CUDA(c, w.t0.ensure((size_t)S * PA * sizeof(double)));
  RSN_CUDA(c, w.tlast.ensure(sd));
  RSN_CUDA(c, w.gcnt.ensure(si));
  RSN_CUDA(c, w.gphase.ensure(si));
  RSN_CUDA(c, w.tgoal.ensure(sd));
  RSN_CUDA(c, w.rgoal.ensure(sd));
  RSN_CUDA(c, w.mu.ensure((size_t)S * PA * sizeof(double2)));
  RSN_CUDA(c, w.rho.ensure((size_t)S * PB * sizeof(double2)));
  RSN_CUDA(c, w.nrm.ensure((size_t)S * PB * sizeof(double)));
  const size_t npj = std::max(1, n_proj);
  RSN_CUDA(c, w.c_r.ensure((size_t)S * npj * sizeof(double2)));
  RSN_CUDA(c, w.c_p.ensure(2 * (size_t)S * npj * sizeof(double2)));
  RSN_CUDA(c, w.c_x.ensure((size_t)S * npj * sizeof(double2)));
  RSN_CUDA(c, w.c_e.ensure((size_t)S * (npj + kCePad) * sizeof(double2)));
  RSN_CUDA(c, cudaMemset(w.c_e.p, 0, (size_t)S * (npj + kCePad) * sizeof(double2)));
  RSN_CUDA(c, w.sched.ensure((3 + 2 * kMaxGraphIters) * sizeof(int)));
  RSN_CUDA(c, w.counters.ensure(4 * sizeof(unsigned long long)));
  RSN_CUDA(c, w.lst.ensure(si));
  RSN_CUDA(c, w.lst_n.ensure(sizeof(int)));
  RSN_CUDA(c, w.inlist.ensure(si));
  RSN_CUDA(c, cudaMemset(w.inlist.p, 0, si));
  RSN_CUDA(c, w.fslot.ensure(si));
  std::vector<long long> hvo(S);
  for (int s = 0; s < S; ++s) hvo[s] = (long long)s * N;
  RSN_CUDA(c, cudaMemcpy(w.voff.p, hvo.data(), sl, cudaMemcpyHostToDevice));
  RSN_CUDA(c, c->bd.ensure(2 * sizeof(BatchDev)));
  w.slots = S;
  w.fp32 = fp32;
  w.N = N;
  w.PA = PA;
  w.PB = PB;
  w.n_proj = n_proj;
  w.generation++;
  clear_graphs(c);
  return RSN_OK;
}

static rsn_status ensure_calls(rsn_ctx* c, long long nsys) {
  CallBufs& q = c->cb;
  const size_t n = (size_t)std::max<long long>(1, nsys);
  RSN_CUDA(c, q.sys_junc.ensure(n * sizeof(int)));
  RSN_CUDA(c, q.sys_E.ensure(n * sizeof(double)));
  RSN_CUDA(c, q.sys_col.ensure(n * sizeof(int)));
  RSN_CUDA(c, q.sys_xo.ensure(n * sizeof(long long)));
  RSN_CUDA(c, q.sys_xfo.ensure(n * sizeof(long long)));
  RSN_CUDA(c, q.sys_dep.ensure(n * sizeof(int)));
  RSN_CUDA(c, q.sys_bn2.ensure(n * sizeof(double)));
  RSN_CUDA(c, q.sys_started.ensure(n * sizeof(int)));
  RSN_CUDA(c, q.out_iters.ensure(n * sizeof(int)));
  RSN_CUDA(c, q.out_relres.ensure(n * sizeof(double)));
  RSN_CUDA(c, q.out_status.ensure(n * sizeof(int)));
  RSN_CUDA(c, q.out_t.ensure(n * sizeof(double)));
  return RSN_OK;
}

// ---------------------------------------------------------------------------
// the streaming solver
// ---------------------------------------------------------------------------
struct StreamIn {
  std::vector<int> junc, col, dep;
  std::vector<double> E, bn2;
  std::vector<long long> xo, xfo;
  void resize(size_t n) {
    junc.assign(n, 0);
    col.assign(n, 0);
    dep.assign(n, -1);
    E.assign(n, 0.0);
    bn2.assign(n, 0.0);
    xo.assign(n, -1);
    xfo.assign(n, 0);
  }
  void push(const StreamIn& o, size_t k) {
    junc.push_back(o.junc[k]);
    col.push_back(o.col[k]);
    dep.push_back(o.dep[k]);
    E.push_back(o.E[k]);
    bn2.push_back(o.bn2[k]);
    xo.push_back(o.xo[k]);
    xfo.push_back(o.xfo[k]);
  }
};
struct StreamOut {
  std::vector<int> iters, status;
  std::vector<double> relres;
  bool timeout = false;
  unsigned long long krylov = 0, updates = 0;
};

// BatchDev view of the slot pool (per-call system queue fields left empty).
static BatchDev slot_batch(rsn_ctx* c, int S, const rsn_solver_opts* o) {
  Workspace& w = c->ws;
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.nslots = S;
  b.PA = w.PA;
  b.PB = w.PB;
  b.state = w.state.as<int>();
  b.sys = w.sys.as<int>();
  b.junc = w.junc.as<int>();
  b.E = w.E.as<double>();
  b.col = w.col.as<int>();
  b.voff = w.voff.as<long long>();
  b.xo = w.xo.as<long long>();
  b.xfo = w.xfo.as<long long>();
  b.iters = w.iters.as<int>();
  b.total_iters = w.total_iters.as<int>();
  b.cyc_iters = w.cyc_iters.as<int>();
  b.n_upd = w.n_upd.as<int>();
  b.restart = w.restart.as<int>();
  b.stall = w.stall.as<int>();
  b.warm = w.warm.as<int>();
  b.rho_cur = w.rho_cur.as<double2>();
  b.beta_cur = w.beta_cur.as<double2>();
  b.bnorm2 = w.bnorm2.as<double>();
  b.sigma = w.sigma.as<double>();
  b.rlast2 = w.rlast2.as<double>();
  b.rrec2 = w.rrec2.as<double>();
  b.tol2 = w.tol2.as<double>();
  b.x64 = w.Xslot.as<double2>();
  b.r = w.r.p;
  b.p0 = w.p0.p;
  b.p1 = w.p1.p;
  b.q = w.q.p;
  b.d = w.d.p;
  b.rho0_part = w.rho0.as<double2>();
  b.nrm0_part = w.nrm0.as<double>();
  b.t0_part = w.t0.as<double>();
  b.tlast = w.tlast.as<double>();
  b.gcnt = w.gcnt.as<int>();
  b.gphase = w.gphase.as<int>();
  b.tgoal = w.tgoal.as<double>();
  b.rgoal = w.rgoal.as<double>();
  b.rho_part = w.rho.as<double2>();
  b.nrm_part = w.nrm.as<double>();
  b.mu_part = w.mu.as<double2>();
  b.c_r = w.c_r.p;
  b.c_p = w.c_p.p;
  b.c_x = w.c_x.as<double2>();
  b.sched = w.sched.as<int>();
  b.counters = w.counters.as<unsigned long long>();
  b.lst = w.lst.as<int>();
  b.lst_n = w.lst_n.as<int>();
  b.inlist = w.inlist.as<int>();
  b.fslot = w.fslot.as<int>();
  b.c_e = w.c_e.p;
  b.ce_stride = std::max(1, c->ws.n_proj) + kCePad;
  b.pstride = c->ws.n_proj;
  b.tol = o->tol;
  b.tol_adj = o->tol_adjoint > 0 ? o->tol_adjoint : o->tol;
  b.tol_T = o->tol_T;
  b.delta = o->tol_inner;
  b.max_iter = o->max_iter;
  b.max_upd = o->max_outer;
  // FP32 cycles end by the cycle cap as well, so that precision-limited systems
  // are seen early; an FP64 cycle runs until its recurrence reaches the target,
  // since true residuals that replace the recurrence in the middle of a slow
  // phase would hide a drifted recurrence
  b.cycle_cap = o->precision == RSN_MIXED ? std::max(32, std::min(o->max_iter, 400)) : std::max(32, o->max_iter);
  b.stall_cap = o->precision == RSN_MIXED ? 3 : 0;
  b.handback = o->precision == RSN_MIXED ? 1 : 0;
  return b;
}

static rsn_status run_stream(rsn_ctx* c, const rsn_solver_opts* o, const StreamIn& in, double2* x64_base,
                             const double2* xf_base, bool want_t, size_t reserved,
                             std::chrono::steady_clock::time_point t_start, StreamOut& out,
                             const ShiftSpec* sh = nullptr, const PoolSpec* pool = nullptr) {
  const long long nsys = (long long)in.E.size();
  const bool fp32 = o->precision == RSN_MIXED;
  const int ns = sh ? sh->n_shift : 0;
  const size_t shift_slot_bytes = sh ? (size_t)ns * sh->nT * sizeof(double2) * (sh->xs_out ? 1 : 2) : 0;
  const int S = choose_slots(c, o, nsys, reserved, shift_slot_bytes, pool ? pool->N : 0);
  rsn_status rs = ensure_ws(c, fp32, S, pool);
  if (rs != RSN_OK) return rs;
  if ((rs = ensure_calls(c, nsys)) != RSN_OK) return rs;
  Workspace& w = c->ws;
  CallBufs& q = c->cb;
  cudaStream_t st = c->st;
  // system queue
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_junc.p, in.junc.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_E.p, in.E.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_col.p, in.col.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_xo.p, in.xo.data(), nsys * sizeof(long long), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_xfo.p, in.xfo.data(), nsys * sizeof(long long), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_dep.p, in.dep.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_bn2.p, in.bn2.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemsetAsync(q.out_status.p, 0xff, nsys * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(q.sys_started.p, 0, nsys * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(q.out_iters.p, 0, nsys * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(q.out_relres.p, 0, nsys * sizeof(double), st));
  if (want_t) RSN_CUDA(c, cudaMemsetAsync(q.out_t.p, 0, nsys * sizeof(double), st));
  // slot pool starts empty
  RSN_CUDA(c, cudaMemsetAsync(w.state.p, 0, S * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.sched.p, 0, (3 + 2 * kMaxGraphIters) * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.counters.p, 0, 4 * sizeof(unsigned long long), st));

  BatchDev b = slot_batch(c, S, o);
  b.x64 = x64_base ? x64_base : w.Xslot.as<double2>();
  b.xf = xf_base;
  b.nsys = (int)nsys;
  b.sys_junc = q.sys_junc.as<int>();
  b.sys_E = q.sys_E.as<double>();
  b.sys_col = q.sys_col.as<int>();
  b.sys_xo = q.sys_xo.as<long long>();
  b.sys_xfo = q.sys_xfo.as<long long>();
  b.sys_dep = q.sys_dep.as<int>();
  b.sys_bn2 = q.sys_bn2.as<double>();
  b.sys_started = q.sys_started.as<int>();
  b.out_iters = q.out_iters.as<int>();
  b.out_relres = q.out_relres.as<double>();
  b.out_status = q.out_status.as<int>();
  b.out_t = want_t ? q.out_t.as<double>() : nullptr;
  if (sh) {
    const size_t nT = (size_t)sh->nT;
    RSN_CUDA(c, q.sh_sig.ensure(ns * sizeof(double)));
    RSN_CUDA(c, q.sh_ps.ensure((size_t)S * ns * nT * sizeof(double2)));
    if (!sh->xs_out) RSN_CUDA(c, q.sh_xs.ensure((size_t)S * ns * nT * sizeof(double2)));
    RSN_CUDA(c, q.sh_pi.ensure(3 * (size_t)S * ns * sizeof(double2)));
    RSN_CUDA(c, q.sh_cit.ensure((size_t)S * ns * sizeof(int)));
    RSN_CUDA(c, q.sh_alpha.ensure(2 * (size_t)S * sizeof(double2)));
    RSN_CUDA(c, q.sh_beta.ensure(2 * (size_t)S * sizeof(double2)));
    RSN_CUDA(c, q.sh_rn2.ensure((size_t)S * sizeof(double)));
    RSN_CUDA(c, q.sh_ts.ensure((size_t)nsys * ns * sizeof(double)));
    RSN_CUDA(c, q.sh_sit.ensure((size_t)nsys * ns * sizeof(int)));
    RSN_CUDA(c, q.sh_srel.ensure((size_t)nsys * ns * sizeof(double)));
    RSN_CUDA(c, cudaMemcpyAsync(q.sh_sig.p, sh->sig.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
    RSN_CUDA(c, cudaMemsetAsync(q.sh_sit.p, 0xff, (size_t)nsys * ns * sizeof(int), st));
    RSN_CUDA(c, cudaMemsetAsync(q.sh_srel.p, 0, (size_t)nsys * ns * sizeof(double), st));
    RSN_CUDA(c, cudaMemsetAsync(q.sh_ts.p, 0, (size_t)nsys * ns * sizeof(double), st));
    b.n_shift = ns;
    b.shift_sig = q.sh_sig.as<double>();
    b.nT = sh->nT;
    b.T_idx = sh->idx;
    if (sh->xs_out) {
      b.xs = sh->xs_out;
      b.xs_by_sys = 1;
      b.xs_sstride = (long long)nT;             // system = column c
      b.xs_estride = sh->n_cols * (long long)nT;  // [n_e][n_cols][N]
    } else {
      b.xs = q.sh_xs.as<double2>();
      b.xs_by_sys = 0;
      b.xs_sstride = (long long)ns * nT;
      b.xs_estride = (long long)nT;
    }
    b.ps = q.sh_ps.as<double2>();
    b.spi = q.sh_pi.as<double2>();
    b.sconv_it = q.sh_cit.as<int>();
    b.salpha = q.sh_alpha.as<double2>();
    b.sbeta = q.sh_beta.as<double2>();
    b.rn2 = q.sh_rn2.as<double>();
    b.out_ts = q.sh_ts.as<double>();
    b.out_sit = q.sh_sit.as<int>();
    b.out_srel = q.sh_srel.as<double>();
  }
  RSN_CUDA(c, cudaMemcpyAsync(c->bd.p, &b, sizeof(b), cudaMemcpyHostToDevice, st));
  const BatchDev* bdev = c->bd.as<BatchDev>();

  LaunchCfg cfg;
  const JuncDev* ji;
  const JuncDev* jr;
  int nB, n_groups, max_np, nS, R;
  bool proj;
  if (pool) {
    ji = pool->ji;
    jr = pool->jr;
    cfg.resid = pool->resid;
    nB = pool->nB;
    proj = pool->n_proj > 0;
    n_groups = pool->n_groups;
    max_np = pool->max_np;
    nS = pool->nS;
    R = pool->R;
  } else {
    if ((rs = make_cfg(c, fp32, S, cfg)) != RSN_OK) return rs;
    ji = cfg.jt_inner;
    jr = cfg.jt_resid;
    nB = c->jh.nB;
    proj = c->n_proj > 0;
    n_groups = c->n_groups;
    max_np = c->max_np;
    nS = c->jh.nS;
    R = c->R;
  }
  const bool multi = pool && pool->K > 1;
  const int ce_stride = b.ce_stride;
  const int KL = std::min(S, kListRows);
  const bool goal = o->tol_T > 0 && !sh;
  const dim3 gr(cfg.resid.n, KL);
  const int G = std::max(1, std::min(kMaxGraphIters, o->graph_iters));
  const bool timing = o->timing != 0;
  while (timing && (int)c->tev.size() < 4 * G) {
    cudaEvent_t e;
    RSN_CUDA(c, cudaEventCreate(&e));
    c->tev.push_back(e);
  }
  // One iteration: the true-residual path of the NEW / CHECK / goal-check slots
  // (list, zero, projections of x, FP64 residual, x update, goal check) runs on
  // the second stream beside the COCG step of the ACTIVE slots (projections of
  // r, operator, update, bookkeeping); both touch disjoint slots.  The
  // scheduler then joins them: finished systems leave, checked systems resume,
  // free slots take queued systems for the next iteration.
  // Shifted systems keep one stream: their per-iteration shift step must see
  // exactly the slots that did a COCG iteration, so the scheduler runs first.
  cudaStream_t st2 = sh ? st : c->st2;
  auto body = [&](int iters, bool capturing) -> cudaError_t {
    // inside stream capture an event record must be an external node to be timeable
    const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.sched.as<int>() + 3 + kMaxGraphIters, 0, iters * sizeof(int), st)) != cudaSuccess)
      return e;
    auto residual_path = [&]() -> cudaError_t {
      cudaError_t e2;
      if ((e2 = launch_list(st2, bdev)) != cudaSuccess) return e2;
      if ((e2 = launch_zero(fp32, KL, nB, st2, jr, bdev)) != cudaSuccess) return e2;
      if (sh && (e2 = launch_shift_init(sh->nT, st2, jr, bdev)) != cudaSuccess) return e2;
      if (proj && (e2 = launch_project(1, fp32, KL, n_groups, max_np, st2, jr, bdev, nullptr, w.c_x.p, multi)) !=
                      cudaSuccess)
        return e2;
      if ((e2 = launch_op(OP_RESID, fp32, R, cfg.resid.ppt, gr, cfg.resid.threads, cfg.resid.smem, st2, jr, bdev,
                          nullptr, nullptr, nullptr)) != cudaSuccess)
        return e2;
      if ((e2 = launch_x_update(fp32, KL, nB, st2, jr, bdev)) != cudaSuccess) return e2;
      if (goal && (e2 = launch_tgoal(st2, jr, bdev)) != cudaSuccess) return e2;
      return cudaSuccess;
    };
    auto schedule = [&](int it) -> cudaError_t {
      cudaError_t e2;
      if ((e2 = launch_sched(S, it, st, jr, bdev)) != cudaSuccess) return e2;
      if ((e2 = launch_emit(S, st, jr, bdev)) != cudaSuccess) return e2;
      if (sh && (e2 = launch_shift_emit(S, ns, st, jr, bdev)) != cudaSuccess) return e2;
      return cudaSuccess;
    };
    for (int it = 0; it < iters; ++it) {
      if (sh) {
        if ((e = residual_path()) != cudaSuccess) return e;
        if ((e = schedule(it)) != cudaSuccess) return e;
      } else {
        if ((e = cudaEventRecord(c->ev_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st2, c->ev_fork, 0)) != cudaSuccess) return e;
        if ((e = residual_path()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->ev_join, st2)) != cudaSuccess) return e;
      }
      // COCG step of the ACTIVE slots (main stream)
      if (proj && (e = launch_project(0, fp32, S, n_groups, max_np, st, ji, bdev, nullptr, w.c_r.p, multi)) !=
                      cudaSuccess)
        return e;
      if (timing && (e = cudaEventRecordWithFlags(c->tev[4 * it], st, evf)) != cudaSuccess) return e;
      if (pool) {
        for (int kd = 0; kd < 4; ++kd)
          if (pool->has[kd] &&
              (e = launch_inner(c, pool->inner[kd], OP_COCG, fp32, S, st, ji, bdev, nullptr, nullptr, nullptr)) !=
                  cudaSuccess)
            return e;
      } else if ((e = launch_inner(c, cfg.inner, OP_COCG, fp32, S, st, ji, bdev, nullptr, nullptr, nullptr)) !=
                 cudaSuccess) {
        return e;
      }
      if (timing && (e = cudaEventRecordWithFlags(c->tev[4 * it + 1], st, evf)) != cudaSuccess) return e;
      if ((e = launch_cocg_update(fp32, S, nB, ce_stride, st, ji, bdev)) != cudaSuccess) return e;
      if (timing && (e = cudaEventRecordWithFlags(c->tev[4 * it + 2], st, evf)) != cudaSuccess) return e;
      if ((e = launch_book(S, it, st, ji, bdev)) != cudaSuccess) return e;
      if (sh && (e = launch_shift_update(S, sh->nT, ns, st, ji, bdev)) != cudaSuccess) return e;
      if (!sh) {
        // join: the scheduler sees both paths of this iteration
        if ((e = cudaStreamWaitEvent(st, c->ev_join, 0)) != cudaSuccess) return e;
        if ((e = schedule(it)) != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  };
  const int per_iter = (proj ? 11 : 9) + (sh ? 3 : 0) + (goal ? 1 : 0);
  const double vbytes = (double)(pool ? pool->N : c->N) * (fp32 ? sizeof(float2) : sizeof(double2));
  cudaGraphExec_t gexec = nullptr;
  if (o->use_graph) {
    GraphKey key{fp32 ? 1 : 0, S, G, w.generation, proj ? 1 : 0, timing ? 1 : 0, ns, (sh ? sh->nT : 0) * 2 + (goal ? 1 : 0)};
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
      gexec = it->second;
    } else {
      cudaGraph_t g = nullptr;
      RSN_CUDA(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = body(G, true);
      cudaError_t e2 = cudaStreamEndCapture(st, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        RSN_FAIL(c, RSN_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      RSN_CUDA(c, cudaGraphInstantiate(&gexec, g, 0));
      cudaGraphDestroy(g);
      c->graphs[key] = gexec;
    }
  }

  // every system needs at most max_iter COCG iterations plus one iteration per
  // true residual, and a dependent system starts after its dependency; this
  // bounds the replays even if the device state were wrong
  const long long waves = (nsys + S - 1) / S;
  bool has_dep = false;
  for (long long k = 0; k < nsys && !has_dep; ++k) has_dep = in.dep[k] >= 0;
  const long long per_sys = (long long)o->max_iter + 2LL * o->max_outer + 8;
  const long long max_replays = ((waves + (has_dep ? 2 : 1)) * per_sys + G) / G + 4;
  bool timeout = false, finished = false, aborted = false;
  const double abort_ratio = fp32 ? 0.5 : 0.0;
  int* hs = c->sched_host;
  const auto t_run = std::chrono::steady_clock::now();
  long long reps_done = 0;
  for (long long rep = 0; rep < max_replays; ++rep) {
    ++reps_done;
    if (gexec) {
      RSN_CUDA(c, cudaGraphLaunch(gexec, st));
    } else {
      RSN_CUDA(c, body(G, false));
    }
    c->st_launches += (int64_t)G * per_iter;
    RSN_CUDA(c, cudaMemcpyAsync(hs, w.sched.p, (3 + 2 * kMaxGraphIters) * sizeof(int), cudaMemcpyDeviceToHost, st));
    RSN_CUDA(c, cudaMemcpyAsync(c->cnt_host, w.counters.p, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                st));
    RSN_CUDA(c, cudaStreamSynchronize(st));
    if (timing) {
      for (int it = 0; it < G; ++it) {
        const int act = hs[3 + kMaxGraphIters + it];
        float m0 = 0.f, m1 = 0.f;
        RSN_CUDA(c, cudaEventElapsedTime(&m0, c->tev[4 * it], c->tev[4 * it + 1]));
        RSN_CUDA(c, cudaEventElapsedTime(&m1, c->tev[4 * it + 1], c->tev[4 * it + 2]));
        if (act == 0) continue;
        c->ks_launches[0]++;
        c->ks_launches[1]++;
        c->ks_ms[0] += m0;
        c->ks_ms[1] += m1;
        c->ks_bytes[0] += 4.0 * vbytes * act;
        c->ks_bytes[1] += 6.0 * vbytes * act;
      }
    }
    if (hs[2] != 0) RSN_FAIL(c, RSN_ECUDA, "a bulk copy did not arrive within its bounded wait (kernel aborted)");
    if (hs[0] >= nsys && hs[1] == 0) {
      finished = true;
      break;
    }
    // mixed precision at a near-resonant energy: once most finished systems were
    // handed back, stop and let the FP64 pass take every remaining system
    if (fp32 && abort_ratio > 0 && c->cnt_host[2] >= (unsigned long long)std::max(32, S / 4) &&
        (double)c->cnt_host[3] > abort_ratio * (double)c->cnt_host[2]) {
      aborted = true;
      break;
    }
    if (o->deadline_ms > 0) {
      const double el_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
      if (el_ms > o->deadline_ms) {
        timeout = true;
        break;
      }
    }
  }
  if (!finished && !timeout && !aborted) RSN_FAIL(c, RSN_ECUDA, "streaming solver exceeded its iteration bound");
  out.iters.resize(nsys);
  out.status.resize(nsys);
  out.relres.resize(nsys);
  unsigned long long cnt[4] = {0, 0, 0, 0};
  RSN_CUDA(c, cudaMemcpyAsync(out.iters.data(), q.out_iters.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(out.status.data(), q.out_status.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(out.relres.data(), q.out_relres.p, nsys * sizeof(double), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(cnt, w.counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaStreamSynchronize(st));
  out.timeout = timeout;
  out.krylov = cnt[0];
  out.updates = cnt[1];
  if (getenv("RSN_VERBOSE")) {
    long long bad = 0, it_max = 0;
    for (long long k = 0; k < nsys; ++k) {
      bad += out.status[k] != 0;
      it_max = std::max<long long>(it_max, out.iters[k]);
    }
    fprintf(stderr, "[rsn] stream %s: %lld systems, %d slots, %lld iterations, %.1f ms, %llu COCG iterations "
            "(max %lld per system), %llu true residuals, %lld unfinished\n", fp32 ? "mixed" : "fp64", nsys, S,
            reps_done * G, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_run).count(),
            (unsigned long long)cnt[0], it_max, (unsigned long long)cnt[1], bad);
  }
  c->st_iters += (int64_t)cnt[0];
  c->st_sweeps += (int64_t)cnt[1];
  return RSN_OK;
}

// classify finished systems into an overall status; fills iters/relres
static rsn_status stream_status(const StreamOut& r, long long n0, long long n, int32_t* iters, double* relres,
                                std::string* why = nullptr) {
  rsn_status worst = RSN_OK;
  long long nbad = 0;
  for (long long k = 0; k < n; ++k) {
    const int stt = r.status[n0 + k];
    const bool ok = stt == 0;
    if (iters) iters[k] = ok ? r.iters[n0 + k] : -std::max(1, r.iters[n0 + k]);
    if (relres) relres[k] = r.relres[n0 + k];
    if (!ok) {
      if (worst == RSN_OK) {
        worst = (stt < 0 || r.timeout) ? RSN_ETIMEOUT : (stt == 2 ? RSN_EBREAKDOWN : RSN_ENOCONV);
        if (why) {
          char buf[256];
          snprintf(buf, sizeof(buf), "system %lld: status %d after %d iterations, relative residual %.3e", n0 + k,
                   stt, r.iters[n0 + k], r.relres[n0 + k]);
          *why = buf;
        }
      }
      ++nbad;
    }
  }
  if (why && nbad) *why += " (" + std::to_string(nbad) + " of " + std::to_string(n) + " systems failed)";
  return worst;
}

static rsn_status check_solve_args(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                   const rsn_solver_opts* o) {
  if (n_e < 0 || n_cols < 0) RSN_FAIL(c, RSN_EINVAL, "negative sizes");
  if ((n_e > 0 && !E) || (n_cols > 0 && !cols) || !o) RSN_FAIL(c, RSN_EINVAL, "NULL argument");
  if (o->precision != RSN_FP64 && o->precision != RSN_MIXED) RSN_FAIL(c, RSN_EINVAL, "bad precision");
  if (!(o->tol > 0) || !(o->tol_adjoint >= 0) || !(o->tol_T >= 0) || !(o->tol_inner > 0) || !(o->tol_inner < 1) || o->max_iter < 1 || o->max_outer < 1 ||
      o->graph_iters < 0 || o->rhs_block < 0)
    RSN_FAIL(c, RSN_EINVAL, "bad solver options");
  for (int e = 0; e < n_e; ++e)
    if (!std::isfinite(E[e])) RSN_FAIL(c, RSN_EINVAL, "E[%d] is not finite", e);
  for (int k = 0; k < n_cols; ++k)
    if (cols[k] < 0 || cols[k] >= c->N) RSN_FAIL(c, RSN_EINVAL, "cols[%d] = %d out of range", k, cols[k]);
  if ((long long)n_e * n_cols >= (1LL << 30)) RSN_FAIL(c, RSN_EINVAL, "too many systems in one call");
  return RSN_OK;
}

static void reset_stats(rsn_ctx* c) {
  c->st_iters = c->st_sweeps = c->st_launches = c->st_fallback = 0;
  for (int k = 0; k < 2; ++k) c->ks_launches[k] = 0, c->ks_ms[k] = 0, c->ks_bytes[k] = 0;
}

// y_k = A(E_k) x_k through the allocating per-call buffers of the context.
static rsn_status apply_impl(rsn_ctx* c, int precision, int n_rhs, const double* E, const void* x_dev, void* y_dev) {
  const bool fp32 = precision == RSN_MIXED;
  CallBufs& q = c->cb;
  // small per-call arrays: E, junction ids, offsets, projections
  RSN_CUDA(c, q.sys_E.ensure(n_rhs * sizeof(double)));
  RSN_CUDA(c, q.sys_junc.ensure(n_rhs * sizeof(int)));
  RSN_CUDA(c, q.sys_xo.ensure(n_rhs * sizeof(long long)));
  RSN_CUDA(c, q.out_t.ensure((size_t)n_rhs * std::max(1, c->n_proj) * sizeof(double2)));
  RSN_CUDA(c, c->bd.ensure(2 * sizeof(BatchDev)));
  std::vector<int> hj(n_rhs, 0);
  std::vector<long long> hvo(n_rhs);
  for (int s = 0; s < n_rhs; ++s) hvo[s] = (long long)s * c->N;
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_E.p, E, n_rhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_junc.p, hj.data(), n_rhs * sizeof(int), cudaMemcpyHostToDevice, c->st));
  RSN_CUDA(c, cudaMemcpyAsync(q.sys_xo.p, hvo.data(), n_rhs * sizeof(long long), cudaMemcpyHostToDevice, c->st));
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.nslots = n_rhs;
  b.junc = q.sys_junc.as<int>();
  b.E = q.sys_E.as<double>();
  b.voff = q.sys_xo.as<long long>();
  b.pstride = c->n_proj;
  RSN_CUDA(c, cudaMemcpyAsync(c->bd.as<BatchDev>() + 1, &b, sizeof(b), cudaMemcpyHostToDevice, c->st));
  const BatchDev* bdev = c->bd.as<BatchDev>() + 1;
  // bulk-copy kernels need 16-byte aligned vectors; otherwise a register tiling
  const bool aligned = (reinterpret_cast<uintptr_t>(x_dev) % 16) == 0 && (reinterpret_cast<uintptr_t>(y_dev) % 16) == 0;
  const Tiling t = choose_tiling(c, !fp32, OP_APPLY, n_rhs, aligned);
  LaunchCfg cfg;
  rsn_status rs = make_cfg(c, t, choose_tiling(c, true, OP_RESID, n_rhs), cfg);
  if (rs != RSN_OK) return rs;
  void* cbuf = q.out_t.p;
  if (c->n_proj > 0)
    RSN_CUDA(c, launch_project(2, fp32, n_rhs, c->n_groups, c->max_np, c->st, cfg.jt_inner, bdev, x_dev, cbuf));
  RSN_CUDA(c, launch_inner(c, t, OP_APPLY, fp32, n_rhs, c->st, cfg.jt_inner, bdev, x_dev, y_dev, cbuf));
  return RSN_OK;
}

extern "C" {

rsn_status rsn_apply(rsn_ctx* c, int precision, int n_rhs, const double* E, const void* x_dev, void* y_dev) {
  if (!c) return RSN_EINVAL;
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if (n_rhs < 0 || (n_rhs > 0 && (!E || !x_dev || !y_dev))) RSN_FAIL(c, RSN_EINVAL, "bad arguments");
  if (n_rhs > kMaxApplyRhs) RSN_FAIL(c, RSN_EINVAL, "n_rhs = %d exceeds %d vectors per call; split the call", n_rhs, kMaxApplyRhs);
  if (precision != RSN_FP64 && precision != RSN_MIXED) RSN_FAIL(c, RSN_EINVAL, "bad precision");
  if (n_rhs == 0) return RSN_OK;
  if ((rs = enter(c)) != RSN_OK) return rs;
  rs = apply_impl(c, precision, n_rhs, E, x_dev, y_dev);
  // the caller's stream is ordered after whatever was queued, also on failure
  const rsn_status rl = leave(c);
  return rs != RSN_OK ? rs : rl;
}

rsn_status rsn_solve_columns(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                             const rsn_solver_opts* o, void* x_dev, int32_t* iters, double* relres) {
  if (!c) return RSN_EINVAL;
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((rs = check_solve_args(c, n_e, E, n_cols, cols, o)) != RSN_OK) return rs;
  const long long nsys = (long long)n_e * n_cols;
  if (nsys == 0) return RSN_OK;
  if (!x_dev) RSN_FAIL(c, RSN_EINVAL, "x_dev is NULL");
  if ((rs = enter(c)) != RSN_OK) return rs;
  reset_stats(c);
  const auto t_start = std::chrono::steady_clock::now();
  RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
  StreamIn in;
  in.resize(nsys);
  for (long long k = 0; k < nsys; ++k) {
    in.E[k] = E[k / n_cols];
    in.col[k] = cols[k % n_cols];
    in.xo[k] = k * c->N;
  }
  StreamOut so;
  if ((rs = run_stream(c, o, in, reinterpret_cast<double2*>(x_dev), nullptr, false, 0, t_start, so)) != RSN_OK)
    return rs;
  if (o->precision == RSN_MIXED) {
    // systems whose FP32 recurrence stalled, or that an aborted mixed pass did
    // not finish, are solved again in FP64 from zero
    std::vector<long long> F;
    StreamIn sub;
    for (long long k = 0; k < nsys; ++k)
      if (so.status[k] != 0) {
        F.push_back(k);
        sub.push(in, (size_t)k);
        sub.bn2.back() = 0.0;  // cold start: a stalled FP32 iterate slows FP64 COCG down
      }
    if (!F.empty()) {
      rsn_solver_opts o64;
      rsn_default_opts(RSN_FP64, &o64);
      o64.tol = o->tol;
      o64.tol_adjoint = o->tol_adjoint;
      o64.tol_T = o->tol_T;
      o64.deadline_ms = o->deadline_ms;
      o64.use_graph = o->use_graph;
      o64.graph_iters = o->graph_iters;
      StreamOut s2;
      if ((rs = run_stream(c, &o64, sub, reinterpret_cast<double2*>(x_dev), nullptr, false, 0, t_start, s2)) !=
          RSN_OK)
        return rs;
      for (size_t f = 0; f < F.size(); ++f) {
        so.status[F[f]] = s2.status[f];
        so.iters[F[f]] += s2.iters[f];
        so.relres[F[f]] = s2.relres[f];
      }
      c->st_fallback += (int64_t)F.size();
    }
  }
  std::string why;
  const rsn_status worst = stream_status(so, 0, nsys, iters, relres, &why);
  RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
  RSN_CUDA(c, cudaEventSynchronize(c->t1));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->t0, c->t1);
  c->st_ms = ms;
  if ((rs = leave(c)) != RSN_OK) return rs;
  if (worst != RSN_OK) RSN_FAIL(c, worst, "some columns did not reach tol: %s", why.c_str());
  return RSN_OK;
}

// Shared driver of the transmission entry points.
//  x_keep (not NULL, T only): the forward columns are written to x_keep
//    [n_e][n_cols][N] (complex128) as well;
//  x_given (not NULL, with dV): the forward columns are taken from x_given
//    [n_e][n_cols][N] and only the adjoint systems are solved;
//  dV (not NULL): vector-Jacobian product sum_e T_bar[e] dT(E[e])/dV_loc.
static rsn_status transmission_impl(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                    const rsn_solver_opts* o, const double* T_bar, double* dV, int dV_dev,
                                    double* T, double2* x_keep = nullptr, const double2* x_given = nullptr) {
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((rs = check_solve_args(c, n_e, E, n_cols, cols, o)) != RSN_OK) return rs;
  const bool adjoint = dV != nullptr;
  const bool reuse = adjoint && x_given != nullptr;
  if (adjoint && n_e > 0 && !T_bar) RSN_FAIL(c, RSN_EINVAL, "T_bar is NULL");
  if ((rs = enter(c)) != RSN_OK) return rs;
  reset_stats(c);
  CallBufs& q = c->cb;
  const long long N = c->N;
  RSN_CUDA(c, q.gr_cols.ensure(std::max(1, n_cols) * sizeof(double)));
  RSN_CUDA(c, q.Td.ensure(std::max(1, n_e) * sizeof(double)));
  if (adjoint) {
    RSN_CUDA(c, q.g.ensure(N * sizeof(double)));
    RSN_CUDA(c, cudaMemsetAsync(q.g.p, 0, N * sizeof(double), c->st));
  }
  std::vector<double> hgr(std::max(1, n_cols));
  for (int k = 0; k < n_cols; ++k) hgr[k] = c->gr[cols[k]];
  RSN_CUDA(c, cudaMemcpyAsync(q.gr_cols.p, hgr.data(), hgr.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  const auto t_start = std::chrono::steady_clock::now();
  RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
  rsn_status worst = RSN_OK;
  std::string why;
  // energies per chunk: the adjoint keeps the solutions of a chunk resident
  // (forward and adjoint: 2 * chunk * n_cols * N complex128; adjoint only when
  // the forward columns are given)
  int chunk = n_e;
  if (adjoint && n_cols > 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const double per_e = (reuse ? 1.0 : 2.0) * n_cols * (double)N * sizeof(double2);
    chunk = (int)std::max(1.0, std::min((double)n_e, 0.45 * (double)fr / per_e));
  }
  for (int e0 = 0; e0 < n_e && n_cols > 0; e0 += chunk) {
    const int ne = std::min(chunk, n_e - e0);
    const long long M = (long long)ne * n_cols;
    // systems: [forward M][adjoint M], [forward M] (T only) or [adjoint M] (reuse)
    const long long F0 = reuse ? 0 : M;      // forward systems
    const long long NS = adjoint ? F0 + M : M;
    StreamIn in;
    in.resize(NS);
    for (long long k = 0; k < F0; ++k) {
      in.E[k] = E[e0 + k / n_cols];
      in.col[k] = cols[k % n_cols];
      in.xo[k] = adjoint ? k * N : (x_keep ? k * N : -1);
    }
    if (adjoint)
      for (long long k = 0; k < M; ++k) {
        in.E[F0 + k] = E[e0 + k / n_cols];
        in.col[F0 + k] = -1;
        in.xo[F0 + k] = (F0 + k) * N;
        in.xfo[F0 + k] = reuse ? (long long)e0 * n_cols * N + k * N : k * N;
        in.dep[F0 + k] = reuse ? -1 : (int)k;
      }
    double2* X = nullptr;
    const double2* XF = nullptr;
    size_t reserved = 0;
    if (adjoint) {
      RSN_CUDA(c, q.X0.ensure((size_t)NS * N * sizeof(double2)));
      X = q.X0.as<double2>();
      XF = reuse ? x_given : X;
    } else if (x_keep) {
      X = x_keep + (size_t)e0 * n_cols * N;
    }
    StreamOut so;
    if ((rs = run_stream(c, o, in, X, XF, true, reserved, t_start, so)) != RSN_OK) return rs;
    RSN_CUDA(c, q.t_all.ensure(NS * sizeof(double)));
    RSN_CUDA(c, cudaMemcpyAsync(q.t_all.p, q.out_t.p, NS * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (o->precision == RSN_MIXED) {
      // systems whose FP32 recurrence stalled (or that the aborted mixed pass
      // never finished) are re-solved in FP64 from zero; an adjoint is redone
      // whenever it or its forward system is
      std::vector<long long> F;
      StreamIn sub;
      std::vector<int> pos(NS, -1);
      for (long long k = 0; k < F0; ++k)
        if (so.status[k] != 0) {
          pos[k] = (int)F.size();
          F.push_back(k);
          sub.push(in, (size_t)k);
          sub.bn2.back() = 0.0;  // cold start (see solve_columns)
        }
      if (adjoint)
        for (long long k = F0; k < NS; ++k)
          if (so.status[k] != 0 || (!reuse && pos[k - F0] >= 0)) {
            F.push_back(k);
            sub.push(in, (size_t)k);
            sub.bn2.back() = 0.0;  // cold start (the right-hand side may have changed)
            sub.dep.back() = reuse ? -1 : pos[k - F0];
          }
      if (!F.empty()) {
        rsn_solver_opts o64;
        rsn_default_opts(RSN_FP64, &o64);
        o64.tol = o->tol;
        o64.tol_adjoint = o->tol_adjoint;
        o64.tol_T = o->tol_T;
        o64.deadline_ms = o->deadline_ms;
        o64.use_graph = o->use_graph;
        o64.graph_iters = o->graph_iters;
        StreamOut s2;
        if ((rs = run_stream(c, &o64, sub, X, XF, true, reserved, t_start, s2)) != RSN_OK) return rs;
        for (size_t f = 0; f < F.size(); ++f) {
          so.status[F[f]] = s2.status[f];
          so.iters[F[f]] += s2.iters[f];
          so.relres[F[f]] = s2.relres[f];
          if (F[f] < F0)
            RSN_CUDA(c, cudaMemcpyAsync(q.t_all.as<double>() + F[f], q.out_t.as<double>() + f, sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->st));
        }
        c->st_fallback += (int64_t)F.size();
      }
    }
    std::string w1;
    rsn_status bs = stream_status(so, 0, NS, nullptr, nullptr, &w1);
    if (worst == RSN_OK && bs != RSN_OK) {
      worst = bs;
      why = (adjoint && !reuse ? "(forward systems 0.." + std::to_string(M - 1) + ", adjoint after) " : std::string()) + w1;
    }
    if (!reuse) {
      RSN_CUDA(c, launch_t_final(ne, n_cols, c->st, q.t_all.as<double>(), q.gr_cols.as<double>(),
                                 q.Td.as<double>() + e0));
      c->st_launches += 1;
    }
    if (adjoint) {
      std::vector<double> hw(M);
      for (long long k = 0; k < M; ++k) hw[k] = 8.0 * c->gr[cols[k % n_cols]] * T_bar[e0 + k / n_cols];
      RSN_CUDA(c, q.wt.ensure(M * sizeof(double)));
      RSN_CUDA(c, cudaMemcpyAsync(q.wt.p, hw.data(), M * sizeof(double), cudaMemcpyHostToDevice, c->st));
      const double2* xfwd = reuse ? x_given + (size_t)e0 * n_cols * N : X;
      RSN_CUDA(c, launch_grad_sys((int)M, N, c->st, X + F0 * N, xfwd, q.wt.as<double>(), q.g.as<double>()));
      c->st_launches += 1;
      RSN_CUDA(c, cudaStreamSynchronize(c->st));  // hw lives on the host stack
    }
  }
  RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
  if (T && n_e > 0 && !reuse) {
    if (n_cols == 0) RSN_CUDA(c, cudaMemsetAsync(q.Td.p, 0, n_e * sizeof(double), c->st));
    RSN_CUDA(c, cudaMemcpyAsync(T, q.Td.p, n_e * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  if (adjoint) {
    RSN_CUDA(c, cudaMemcpyAsync(dV, q.g.p, N * sizeof(double), dV_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->st));
  }
  RSN_CUDA(c, cudaStreamSynchronize(c->st));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->t0, c->t1);
  c->st_ms = ms;
  if ((rs = leave(c)) != RSN_OK) return rs;
  if (worst != RSN_OK) RSN_FAIL(c, worst, "some systems did not reach tol: %s", why.c_str());
  return RSN_OK;
}

rsn_status rsn_transmission(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                            const rsn_solver_opts* o, double* T) {
  if (!c) return RSN_EINVAL;
  if (n_e > 0 && !T) RSN_FAIL(c, RSN_EINVAL, "T is NULL");
  return transmission_impl(c, n_e, E, n_cols, cols, o, nullptr, nullptr, 0, T);
}

rsn_status rsn_transmission_vjp(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                const rsn_solver_opts* o, const double* T_bar, double* dV, int dV_is_device,
                                double* T) {
  if (!c) return RSN_EINVAL;
  if (!dV) RSN_FAIL(c, RSN_EINVAL, "dV is NULL");
  return transmission_impl(c, n_e, E, n_cols, cols, o, T_bar, dV, dV_is_device, T);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Block COCG: the columns of one energy in blocks of B share one block Krylov
// space.  Each block runs FP64 outer steps (defect correction):
//   R = b - A X (FP64), ||r_j||, t_j = sum_L Gamma_L |x_j|^2
//   column j is done when ||r_j|| <= tol and (tol_T > 0) the change of t_j made
//   by the last correction, scaled by ten times that step's residual
//   reduction, is at most tol_T t_j (the t_j error of the new iterate shrinks
//   with its residual)
//   A D = R / ||R|| column-wise by the FP32 block recurrence (block_kernels.cu)
//   until every column's recurrence residual fell by tol_inner
//   X += ||R|| D
// Blocks finish independently; the kernels of a step run over the listed
// (active) blocks only.
// ---------------------------------------------------------------------------
namespace {
struct BlkRun {
  int B = 0, nbw = 0, S = 0;
  std::vector<int> act;  // active blocks (wave-local)
};
}  // namespace

// Upload the block list and the apply lists (members of the listed blocks).
static rsn_status blk_set_lists(rsn_ctx* c, const BlkRun& br, const std::vector<int>& list,
                                const std::vector<double>& memE) {
  BlkBufs& q = c->bb;
  const int B = br.B;
  const int nm = (int)list.size() * B;
  std::vector<long long> vo(std::max(1, nm));
  std::vector<double> ve(std::max(1, nm));
  for (size_t u = 0; u < list.size(); ++u)
    for (int a = 0; a < B; ++a) {
      const int v = list[u] * B + a;
      vo[u * B + a] = (long long)v * c->N;
      ve[u * B + a] = memE[v];
    }
  if (!list.empty()) {
    RSN_CUDA(c, cudaMemcpyAsync(q.blist.p, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, cudaMemcpyAsync(q.voff.p, vo.data(), nm * sizeof(long long), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, cudaMemcpyAsync(q.vE.p, ve.data(), nm * sizeof(double), cudaMemcpyHostToDevice, c->st));
  }
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.nslots = nm;
  b.junc = q.vjunc.as<int>();
  b.E = q.vE.as<double>();
  b.voff = q.voff.as<long long>();
  b.pstride = c->n_proj;
  b.sched = q.stat.as<int>();  // [2]: an operator kernel's bounded wait gave up
  RSN_CUDA(c, cudaMemcpyAsync(q.bdev.p, &b, sizeof(b), cudaMemcpyHostToDevice, c->st));
  // pageable sources: the copies above are staged before they return
  return RSN_OK;
}

// y = A(E) x over the listed members (projections first, then the operator)
static rsn_status blk_apply(rsn_ctx* c, const Tiling& t, const JuncDev* jt, bool fp32, int nm, const void* x,
                            void* y) {
  BlkBufs& q = c->bb;
  const BatchDev* bd = q.bdev.as<BatchDev>();
  if (c->n_proj > 0)
    RSN_CUDA(c, launch_project(2, fp32, nm, c->n_groups, c->max_np, c->st, jt, bd, x, q.cbuf.p));
  RSN_CUDA(c, launch_inner(c, t, OP_APPLY, fp32, nm, c->st, jt, bd, x, y, q.cbuf.p));
  c->st_launches += c->n_proj > 0 ? 2 : 1;
  return RSN_OK;
}

static rsn_status block_impl(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols, int B,
                             double tol_in, const rsn_solver_opts* o, double2* x_out, double* t_out, double* T,
                             int32_t* iters, double* relres) {
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((rs = check_solve_args(c, n_e, E, n_cols, cols, o)) != RSN_OK) return rs;
  if (B != 4 && B != 8 && B != 16) RSN_FAIL(c, RSN_EINVAL, "block = %d: must be 4, 8 or 16", B);
  if (o->precision != RSN_MIXED)
    RSN_FAIL(c, RSN_EINVAL, "the block recurrence runs in complex FP32 under FP64 refinement: precision must be RSN_MIXED");
  if (tol_in == 0.0) tol_in = 1e-4;
  if (!(tol_in > 0.0 && tol_in < 1.0)) RSN_FAIL(c, RSN_EINVAL, "tol_inner must lie in (0, 1) (0: default 1e-4)");
  const long long N = c->N;
  if (N < 2 * B) RSN_FAIL(c, RSN_EINVAL, "grid of %lld points is too small for blocks of %d", N, B);
  {
    std::vector<int32_t> sc(cols, cols + n_cols);
    std::sort(sc.begin(), sc.end());
    for (int k = 1; k < n_cols; ++k)
      if (sc[k] == sc[k - 1]) RSN_FAIL(c, RSN_EINVAL, "column %d appears twice (a block needs distinct columns)", sc[k]);
  }
  if ((rs = enter(c)) != RSN_OK) return rs;
  // every exit after enter() orders the caller's stream after the queued work
  auto run = [&]() -> rsn_status {
    reset_stats(c);
    BlkBufs& q = c->bb;
    const auto t_start = std::chrono::steady_clock::now();
    RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
    // padding members of a short last block: grid points outside the column set
    std::vector<int> pad;
    {
      std::vector<int32_t> sc(cols, cols + n_cols);
      std::sort(sc.begin(), sc.end());
      for (long long i = 0; i < N && (int)pad.size() < B; ++i)
        if (!std::binary_search(sc.begin(), sc.end(), (int32_t)i)) pad.push_back((int)i);
      if ((int)pad.size() < (B - n_cols % B) % B)
        RSN_FAIL(c, RSN_EINVAL, "too few grid points outside the column set to pad the last block");
    }
    const int nbe = (n_cols + B - 1) / B;  // blocks per energy
    const long long nb = (long long)n_e * nbe;
    std::vector<double> t_host((size_t)std::max(1, n_e) * std::max(1, n_cols), 0.0);
    rsn_status worst = RSN_OK;
    long long n_fail = 0, n_brk = 0, n_late = 0, n_hand = 0;
    const size_t per_member = (size_t)N * (4 * sizeof(float2) + 2 * sizeof(double2)) + 4096;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    // members per wave: within memory and within a launch's grid.y (one CTA row per member)
    const long long cap = std::max<long long>(
        1, std::min<long long>(kMaxApplyRhs / B, (long long)(0.5 * (double)fr / ((double)per_member * B))));
    for (long long b0 = 0; b0 < nb; b0 += cap) {
      BlkRun br;
      br.B = B;
      br.nbw = (int)std::min<long long>(cap, nb - b0);
      br.S = br.nbw * B;
      const int nbw = br.nbw, S = br.S;
      // members: E, column, real (output index) or padding (-1)
      std::vector<double> memE(S);
      std::vector<int> memCol(S);
      std::vector<long long> memOut(S);
      for (int k = 0; k < nbw; ++k) {
        const long long gb = b0 + k;
        const int e = (int)(gb / nbe), cb = (int)(gb % nbe);
        int np = 0;
        for (int a = 0; a < B; ++a) {
          const int kc = cb * B + a;
          const int v = k * B + a;
          memE[v] = E[e];
          if (kc < n_cols) {
            memCol[v] = cols[kc];
            memOut[v] = (long long)e * n_cols + kc;
          } else {
            memCol[v] = pad[np++];
            memOut[v] = -1;
          }
        }
      }
      // buffers
      const size_t vb32 = (size_t)S * N * sizeof(float2), vb64 = (size_t)S * N * sizeof(double2);
      RSN_CUDA(c, q.W.ensure(vb32));
      RSN_CUDA(c, q.P.ensure(vb32));
      RSN_CUDA(c, q.AP.ensure(vb32));
      RSN_CUDA(c, q.D.ensure(vb32));
      RSN_CUDA(c, q.X.ensure(vb64));
      RSN_CUDA(c, q.R.ensure(vb64));
      int nchunk = std::max(1, std::min(64, (4 * 152 + nbw - 1) / nbw));
      long long chunk_pts = (N + nchunk - 1) / nchunk;
      chunk_pts = (chunk_pts + kBlkTile - 1) / kBlkTile * kBlkTile;
      nchunk = (int)((N + chunk_pts - 1) / chunk_pts);
      int nchunkR = std::max(1, std::min(32, (8 * 152 + S - 1) / S));
      long long chunkR_pts = (N + nchunkR - 1) / nchunkR;
      nchunkR = (int)((N + chunkR_pts - 1) / chunkR_pts);
      const size_t bb2 = (size_t)nbw * B * B;
      RSN_CUDA(c, q.part.ensure((size_t)nbw * nchunk * 2 * B * B * sizeof(double2)));
      RSN_CUDA(c, q.xi.ensure(bb2 * sizeof(double2)));
      RSN_CUDA(c, q.QQ.ensure(bb2 * sizeof(double2)));
      RSN_CUDA(c, q.xi0n.ensure((size_t)S * sizeof(double)));
      RSN_CUDA(c, q.alpha.ensure(bb2 * sizeof(float2)));
      RSN_CUDA(c, q.axi.ensure(bb2 * sizeof(float2)));
      RSN_CUDA(c, q.tinv.ensure(bb2 * sizeof(float2)));
      RSN_CUDA(c, q.tinv64.ensure(bb2 * sizeof(double2)));
      RSN_CUDA(c, q.beta.ensure(bb2 * sizeof(float2)));
      RSN_CUDA(c, q.flag.ensure((size_t)nbw * sizeof(int)));
      RSN_CUDA(c, q.its.ensure((size_t)nbw * sizeof(int)));
      RSN_CUDA(c, q.rpart.ensure((size_t)S * nchunkR * 2 * sizeof(double)));
      RSN_CUDA(c, q.rn.ensure((size_t)S * sizeof(double)));
      RSN_CUDA(c, q.tt.ensure((size_t)S * sizeof(double)));
      RSN_CUDA(c, q.blist.ensure((size_t)nbw * sizeof(int)));
      RSN_CUDA(c, q.col.ensure((size_t)S * sizeof(int)));
      RSN_CUDA(c, q.vE.ensure((size_t)S * sizeof(double)));
      RSN_CUDA(c, q.vjunc.ensure((size_t)S * sizeof(int)));
      RSN_CUDA(c, q.voff.ensure((size_t)S * sizeof(long long)));
      RSN_CUDA(c, q.cbuf.ensure((size_t)S * std::max(1, c->n_proj) * sizeof(double2)));
      RSN_CUDA(c, q.dev.ensure(sizeof(BlkDev)));
      RSN_CUDA(c, q.bdev.ensure(sizeof(BatchDev)));
      RSN_CUDA(c, q.jd.ensure(2 * sizeof(JuncDev)));
      RSN_CUDA(c, q.stat.ensure(4 * sizeof(int)));
      RSN_CUDA(c, cudaMemsetAsync(q.stat.p, 0, 4 * sizeof(int), c->st));
      RSN_CUDA(c, cudaMemsetAsync(q.vjunc.p, 0, (size_t)S * sizeof(int), c->st));
      RSN_CUDA(c, cudaMemsetAsync(q.X.p, 0, vb64, c->st));
      RSN_CUDA(c, cudaMemsetAsync(q.flag.p, 0, (size_t)nbw * sizeof(int), c->st));
      RSN_CUDA(c, cudaMemcpyAsync(q.col.p, memCol.data(), (size_t)S * sizeof(int), cudaMemcpyHostToDevice, c->st));
      BlkDev hd;
      memset(&hd, 0, sizeof(hd));
      hd.B = B;
      hd.N = N;
      hd.nchunk = nchunk;
      hd.chunk_pts = chunk_pts;
      hd.nchunkR = nchunkR;
      hd.chunkR_pts = chunkR_pts;
      RSN_CUDA(c, q.icap.ensure((size_t)nbw * sizeof(int)));
      hd.icap = q.icap.as<int>();
      hd.tol_in = tol_in;
      hd.blist = q.blist.as<int>();
      hd.col = q.col.as<int>();
      hd.gl = c->gld.as<double>();
      hd.xi = q.xi.as<double2>();
      hd.QQ = q.QQ.as<double2>();
      hd.xi0n = q.xi0n.as<double>();
      hd.part = q.part.as<double2>();
      hd.alpha = q.alpha.as<float2>();
      hd.axi = q.axi.as<float2>();
      hd.tinv = q.tinv.as<float2>();
      hd.tinv64 = q.tinv64.as<double2>();
      hd.beta = q.beta.as<float2>();
      hd.flag = q.flag.as<int>();
      hd.its = q.its.as<int>();
      hd.W = q.W.as<float2>();
      hd.P = q.P.as<float2>();
      hd.AP = q.AP.as<float2>();
      hd.D = q.D.as<float2>();
      hd.X = q.X.as<double2>();
      hd.R = q.R.as<double2>();
      hd.rpart = q.rpart.as<double>();
      hd.rn = q.rn.as<double>();
      hd.tt = q.tt.as<double>();
      RSN_CUDA(c, cudaMemcpyAsync(q.dev.p, &hd, sizeof(hd), cudaMemcpyHostToDevice, c->st));
      const BlkDev* dd = q.dev.as<BlkDev>();
      // operator tilings: FP32 apply of P, FP64 apply of X
      const bool al32 = (N * (long long)sizeof(float2)) % 16 == 0;
      const Tiling t32 = choose_tiling(c, false, OP_APPLY, S, al32);
      const Tiling t64 = choose_tiling(c, true, OP_APPLY, S, false);
      {
        JuncDev js[2] = {c->jh, c->jh};
        const Tiling* tt2[2] = {&t32, &t64};
        for (int k = 0; k < 2; ++k) {
          const Tiling& t = *tt2[k];
          js[k].TY = t.TY;
          js[k].Lz = t.Lz;
          js[k].ytiles = t.ytiles;
          js[k].ztiles = t.ztiles;
          js[k].nA = t.n;
          js[k].nR = t.n;
          js[k].kind = t.plane ? kOpPlane : t.pair ? kOpPair : t.tma ? kOpTma : kOpReg;
        }
        RSN_CUDA(c, cudaMemcpyAsync(q.jd.p, js, 2 * sizeof(JuncDev), cudaMemcpyHostToDevice, c->st));
      }
      const JuncDev* j32 = q.jd.as<JuncDev>();
      const JuncDev* j64 = q.jd.as<JuncDev>() + 1;
      // outer loop
      std::vector<int> act(nbw);
      for (int k = 0; k < nbw; ++k) act[k] = k;
      std::vector<double> rn(S), tt(S), rn_prev(S, 1.0), t_prev(S, 0.0), dt_prev(S, HUGE_VAL);
      std::vector<long long> apps(nbw, 0);
      std::vector<int> stall(nbw, 0), failed(nbw, 0), flags(nbw), its(nbw);
      // Inner iteration cap per block: the first inner solve (from the unit
      // columns) may take up to min(max_iter, kBlkInnerCap); a restart that runs
      // past twice the first solve's count has lost its block's orthogonality
      // (FP32 Gram matrices of nearly dependent residual directions) and is
      // abandoned, the block going to the plain solver.
      std::vector<int> icap(nbw, std::min(o->max_iter, kBlkInnerCap));
      for (int outer = 0;; ++outer) {
        if (o->deadline_ms > 0) {
          const double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
          if (el > o->deadline_ms) {
            for (int k : act) failed[k] = 2;
            break;
          }
        }
        if (outer > 0) {
          // an inner solve that hit its cap or broke down leaves a correction of
          // unknown quality: its block keeps its last FP64 iterate and goes to the
          // plain solver
          std::vector<int> good;
          for (int k : act)
            if (flags[k] == 1) good.push_back(k);
            else failed[k] = 1;
          act.swap(good);
          if (act.empty()) break;
        }
        const int na = (int)act.size();
        if ((rs = blk_set_lists(c, br, act, memE)) != RSN_OK) return rs;
        if (outer > 0) {
          RSN_CUDA(c, launch_blk_xupd(B, na, c->st, dd, N));
          if ((rs = blk_apply(c, t64, j64, false, na * B, q.X.p, q.R.p)) != RSN_OK) return rs;
          for (int k : act) apps[k] += 1;
        }
        RSN_CUDA(c, launch_blk_resid(B, na, nchunkR, outer > 0, c->st, dd));
        RSN_CUDA(c, launch_blk_norm(B, na, nchunkR, c->st, dd));
        c->st_launches += outer > 0 ? 3 : 2;
        RSN_CUDA(c, cudaMemcpyAsync(rn.data(), q.rn.p, (size_t)S * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        RSN_CUDA(c, cudaMemcpyAsync(tt.data(), q.tt.p, (size_t)S * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        int hstat[4] = {0, 0, 0, 0};
        RSN_CUDA(c, cudaMemcpyAsync(hstat, q.stat.p, sizeof(hstat), cudaMemcpyDeviceToHost, c->st));
        RSN_CUDA(c, cudaStreamSynchronize(c->st));
        if (hstat[2]) RSN_FAIL(c, RSN_ETIMEOUT, "an operator kernel gave up waiting for a bulk copy");
        std::vector<int> keep;
        for (int k : act) {
          bool all = true, progress = false;
          for (int a = 0; a < B; ++a) {
            const int v = k * B + a;
            if (memOut[v] < 0) continue;
            bool ok = std::isfinite(rn[v]) && rn[v] <= o->tol;
            if (ok && o->tol_T > 0.0) {
              if (outer < 2) {
                ok = false;
              } else {
                const double dt = std::fabs(tt[v] - t_prev[v]);
                const double red = std::min(1.0, 10.0 * rn[v] / std::max(rn_prev[v], 1e-300));
                ok = dt * red <= o->tol_T * tt[v] || dt == 0.0;
              }
            }
            if (!ok) all = false;
            // progress: the residual halved, or (at the residual target) the T
            // partial's change halved
            const double dt = std::fabs(tt[v] - t_prev[v]);
            if (outer == 0 || rn[v] < 0.5 * rn_prev[v] || (rn[v] <= o->tol && dt < 0.5 * dt_prev[v])) progress = true;
          }
          for (int a = 0; a < B; ++a) {
            const int v = k * B + a;
            if (outer > 0) dt_prev[v] = std::fabs(tt[v] - t_prev[v]);
            rn_prev[v] = rn[v];
            t_prev[v] = tt[v];
          }
          if (all) continue;
          stall[k] = progress ? 0 : stall[k] + 1;
          if (stall[k] >= 3 || outer >= o->max_outer) {
            failed[k] = 1;
            continue;
          }
          keep.push_back(k);
        }
        act.swap(keep);
        if (act.empty()) break;
        // inner solve on the normalised residual block
        const int na2 = (int)act.size();
        if ((rs = blk_set_lists(c, br, act, memE)) != RSN_OK) return rs;
        // the previous inner solve left its end state in the flags; the kernels
        // of the new one (the Gram of W_0 first) run only on unflagged blocks
        RSN_CUDA(c, cudaMemsetAsync(q.flag.p, 0, (size_t)nbw * sizeof(int), c->st));
        RSN_CUDA(c, cudaMemcpyAsync(q.icap.p, icap.data(), (size_t)nbw * sizeof(int), cudaMemcpyHostToDevice, c->st));
        RSN_CUDA(c, launch_blk_scale(B, na2, c->st, dd, N));
        RSN_CUDA(c, launch_blk_gram64(B, na2, nchunk, c->st, dd));
        RSN_CUDA(c, launch_blk_small(B, 0, na2, c->st, dd));
        RSN_CUDA(c, launch_blk_q0(B, na2, c->st, dd, N));
        c->st_launches += 4;
        std::vector<int> in = act;
        const int kChunk = 8;
        while (!in.empty()) {
          const int ni = (int)in.size();
          for (int it = 0; it < kChunk; ++it) {
            RSN_CUDA(c, launch_blk_comb_p(B, ni, c->st, dd, N));
            if ((rs = blk_apply(c, t32, j32, true, ni * B, q.P.p, q.AP.p)) != RSN_OK) return rs;
            RSN_CUDA(c, launch_blk_gram(B, 0, ni, nchunk, c->st, dd));
            RSN_CUDA(c, launch_blk_small(B, 1, ni, c->st, dd));
            RSN_CUDA(c, launch_blk_comb_w(B, ni, c->st, dd, N));
            RSN_CUDA(c, launch_blk_gram(B, 1, ni, nchunk, c->st, dd));
            RSN_CUDA(c, launch_blk_small(B, 2, ni, c->st, dd));
            c->st_launches += 6;
          }
          RSN_CUDA(c, cudaMemcpyAsync(flags.data(), q.flag.p, (size_t)nbw * sizeof(int), cudaMemcpyDeviceToHost, c->st));
          RSN_CUDA(c, cudaStreamSynchronize(c->st));
          std::vector<int> nxt;
          for (int k : in)
            if (flags[k] == 0) nxt.push_back(k);
          if (nxt.size() != in.size()) {
            in.swap(nxt);
            if (!in.empty() && (rs = blk_set_lists(c, br, in, memE)) != RSN_OK) return rs;
          }
        }
        RSN_CUDA(c, cudaMemcpyAsync(its.data(), q.its.p, (size_t)nbw * sizeof(int), cudaMemcpyDeviceToHost, c->st));
        RSN_CUDA(c, cudaStreamSynchronize(c->st));
        for (int k : act) {
          apps[k] += its[k];
          if (flags[k] == 2) ++n_brk;
          if (outer == 0) icap[k] = std::min(icap[k], std::max(64, 2 * its[k]));
        }
      }
      // Blocks that did not finish: their columns go to the plain slot-pool
      // solver (FP32 recurrence with FP64 reliable updates and its own FP64
      // re-solve of stalled systems), warm-started from the block's last FP64
      // iterate.
      std::vector<int> hv;
      for (int k = 0; k < nbw; ++k)
        if (failed[k] == 1)
          for (int a = 0; a < B; ++a)
            if (memOut[k * B + a] >= 0) hv.push_back(k * B + a);
      std::vector<int> hst(S, 0), hit(S, 0);
      if (!hv.empty()) {
        const int nh = (int)hv.size();
        StreamIn in;
        in.resize(nh);
        for (int u = 0; u < nh; ++u) {
          in.E[u] = memE[hv[u]];
          in.col[u] = memCol[hv[u]];
          in.xo[u] = (long long)hv[u] * N;
          in.bn2[u] = 1.0;  // ||e_col||^2: start from the iterate in X
        }
        StreamOut so;
        if ((rs = run_stream(c, o, in, q.X.as<double2>(), nullptr, true, 0, t_start, so)) != RSN_OK) return rs;
        std::vector<double> th(nh);
        RSN_CUDA(c, cudaMemcpyAsync(th.data(), c->cb.out_t.p, nh * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        RSN_CUDA(c, cudaStreamSynchronize(c->st));
        std::vector<int> F;
        StreamIn sub;
        for (int u = 0; u < nh; ++u) {
          const int v = hv[u];
          tt[v] = th[u];
          rn[v] = so.relres[u];
          hit[v] = so.iters[u];
          hst[v] = so.status[u];
          if (so.status[u] != 0 && o->precision == RSN_MIXED) {
            F.push_back(u);
            sub.push(in, (size_t)u);
            sub.bn2.back() = 0.0;  // cold start: a stalled FP32 iterate slows FP64 COCG down
          }
        }
        if (!F.empty()) {
          rsn_solver_opts o64;
          rsn_default_opts(RSN_FP64, &o64);
          o64.tol = o->tol;
          o64.tol_T = o->tol_T;
          o64.deadline_ms = o->deadline_ms;
          StreamOut s2;
          if ((rs = run_stream(c, &o64, sub, q.X.as<double2>(), nullptr, true, 0, t_start, s2)) != RSN_OK) return rs;
          std::vector<double> t2(F.size());
          RSN_CUDA(c, cudaMemcpyAsync(t2.data(), c->cb.out_t.p, F.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                      c->st));
          RSN_CUDA(c, cudaStreamSynchronize(c->st));
          for (size_t f = 0; f < F.size(); ++f) {
            const int v = hv[F[f]];
            tt[v] = t2[f];
            rn[v] = s2.relres[f];
            hit[v] += s2.iters[f];
            hst[v] = s2.status[f];
          }
        }
        n_hand += nh;
      }
      // outputs of the real members
      for (int k = 0; k < nbw; ++k) {
        if (failed[k] == 2) ++n_late;
        for (int a = 0; a < B; ++a) {
          const int v = k * B + a;
          const long long out = memOut[v];
          if (out < 0) continue;
          t_host[out] = tt[v];
          if (t_out) t_out[out] = tt[v];
          const bool bad = failed[k] == 2 || (failed[k] == 1 && hst[v] != 0);
          if (bad && failed[k] == 1) ++n_fail;
          if (iters) iters[out] = bad ? -1 : (int32_t)std::min<long long>(apps[k] + hit[v], INT32_MAX);
          if (relres) relres[out] = rn[v];
          c->st_iters += apps[k];
          if (x_out)
            RSN_CUDA(c, cudaMemcpyAsync(x_out + out * N, q.X.as<double2>() + (size_t)v * N, N * sizeof(double2),
                                        cudaMemcpyDeviceToDevice, c->st));
        }
      }
    }
    if (n_fail > 0) worst = RSN_ENOCONV;
    if (n_late > 0) worst = RSN_ETIMEOUT;
    if (T && n_e > 0) {
      RSN_CUDA(c, q.t_all.ensure(t_host.size() * sizeof(double)));
      RSN_CUDA(c, q.gr_cols.ensure(std::max(1, n_cols) * sizeof(double)));
      RSN_CUDA(c, q.Td.ensure(n_e * sizeof(double)));
      std::vector<double> hgr(std::max(1, n_cols));
      for (int k = 0; k < n_cols; ++k) hgr[k] = c->gr[cols[k]];
      RSN_CUDA(c, cudaMemcpyAsync(q.t_all.p, t_host.data(), t_host.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      RSN_CUDA(c, cudaMemcpyAsync(q.gr_cols.p, hgr.data(), hgr.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      if (n_cols > 0) {
        RSN_CUDA(c, launch_t_final(n_e, n_cols, c->st, q.t_all.as<double>(), q.gr_cols.as<double>(), q.Td.as<double>()));
        c->st_launches += 1;
      } else {
        RSN_CUDA(c, cudaMemsetAsync(q.Td.p, 0, n_e * sizeof(double), c->st));
      }
      RSN_CUDA(c, cudaMemcpyAsync(T, q.Td.p, n_e * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
    RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
    RSN_CUDA(c, cudaStreamSynchronize(c->st));
    float ms = 0;
    cudaEventElapsedTime(&ms, c->t0, c->t1);
    c->st_ms = ms;
    c->st_fallback = n_hand;
    (void)n_brk;
    if (worst != RSN_OK)
      RSN_FAIL(c, worst, "%lld columns did not reach tol / tol_T, %lld blocks stopped at the deadline", n_fail, n_late);
    return RSN_OK;
  };
  rs = run();
  const rsn_status rl = leave(c);
  return rs != RSN_OK ? rs : rl;
}

extern "C" {

rsn_status rsn_solve_columns_block(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols, int block,
                                   double tol_inner, const rsn_solver_opts* o, void* x_dev, double* t_cols,
                                   int32_t* iters, double* relres) {
  if (!c) return RSN_EINVAL;
  if ((long long)n_e * n_cols > 0 && !x_dev) RSN_FAIL(c, RSN_EINVAL, "x_dev is NULL");
  return block_impl(c, n_e, E, n_cols, cols, block, tol_inner, o, reinterpret_cast<double2*>(x_dev), t_cols, nullptr,
                    iters, relres);
}

rsn_status rsn_transmission_block(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols, int block,
                                  double tol_inner, const rsn_solver_opts* o, double* T, double* t_cols,
                                  int32_t* iters) {
  if (!c) return RSN_EINVAL;
  if (n_e > 0 && !T) RSN_FAIL(c, RSN_EINVAL, "T is NULL");
  return block_impl(c, n_e, E, n_cols, cols, block, tol_inner, o, nullptr, t_cols, T, iters, nullptr);
}

}  // extern "C"

// Shared driver of the shifted entry points: one seed system per column at
// the energy nearest the middle of the window; every energy is a shift of it.
// Shifts that did not converge within max_iter seed iterations are solved
// again one by one by the plain FP64 path.  full: every grid point tracked,
// iterates written to x_dev [n_e][n_cols][N]; else the Gamma_L support only
// and T[e] = 4 sum_c Gamma_R,c t_{e,c}.
static rsn_status shifted_impl(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                               const rsn_solver_opts* o, void* x_dev, int32_t* iters, double* relres, double* T) {
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((rs = check_solve_args(c, n_e, E, n_cols, cols, o)) != RSN_OK) return rs;
  if (o->precision != RSN_FP64)
    RSN_FAIL(c, RSN_EINVAL, "shifted solves run in FP64: the mixed mode's true-residual replacements would break "
                            "the collinearity of the shifted residuals");
  const bool full = x_dev != nullptr;
  const long long nsys = n_cols;
  if (n_e == 0 || n_cols == 0) {
    if (T) for (int e = 0; e < n_e; ++e) T[e] = 0.0;
    return RSN_OK;
  }
  if (!full && c->nL == 0) RSN_FAIL(c, RSN_EINVAL, "Gamma_L is zero everywhere: no transmission to track");
  if ((rs = enter(c)) != RSN_OK) return rs;
  reset_stats(c);
  CallBufs& q = c->cb;
  const long long N = c->N;
  const auto t_start = std::chrono::steady_clock::now();
  RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
  // seed: the energy nearest the middle of the window
  double lo = E[0], hi = E[0];
  for (int e = 1; e < n_e; ++e) lo = std::min(lo, E[e]), hi = std::max(hi, E[e]);
  int seed = 0;
  for (int e = 1; e < n_e; ++e)
    if (std::fabs(E[e] - 0.5 * (lo + hi)) < std::fabs(E[seed] - 0.5 * (lo + hi))) seed = e;
  ShiftSpec sh;
  sh.n_shift = n_e;
  sh.sig.resize(n_e);
  for (int e = 0; e < n_e; ++e) sh.sig[e] = E[e] - E[seed];
  sh.n_cols = n_cols;
  if (full) {
    std::vector<int> all(N);
    for (long long i = 0; i < N; ++i) all[i] = (int)i;
    RSN_CUDA(c, q.sh_idx.ensure(N * sizeof(int)));
    RSN_CUDA(c, cudaMemcpyAsync(q.sh_idx.p, all.data(), N * sizeof(int), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, cudaStreamSynchronize(c->st));  // `all` lives on the host stack
    sh.idx = q.sh_idx.as<int>();
    sh.nT = (int)N;
    sh.xs_out = reinterpret_cast<double2*>(x_dev);
  } else {
    sh.idx = c->L_idx.as<int>();
    sh.nT = c->nL;
  }
  StreamIn in;
  in.resize(nsys);
  for (long long k = 0; k < nsys; ++k) {
    in.E[k] = E[seed];
    in.col[k] = cols[k];
    in.xo[k] = -1;  // the seed's own iterate stays in slot storage
  }
  StreamOut so;
  if ((rs = run_stream(c, o, in, nullptr, nullptr, false, 0, t_start, so, &sh)) != RSN_OK) return rs;
  const size_t ne_c = (size_t)n_e * n_cols;
  std::vector<int> sit(ne_c);
  std::vector<double> srel(ne_c);
  RSN_CUDA(c, cudaMemcpyAsync(sit.data(), q.sh_sit.p, ne_c * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  RSN_CUDA(c, cudaMemcpyAsync(srel.data(), q.sh_srel.p, ne_c * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  RSN_CUDA(c, q.t_all.ensure(ne_c * sizeof(double)));
  RSN_CUDA(c, cudaMemcpyAsync(q.t_all.p, q.sh_ts.p, ne_c * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  RSN_CUDA(c, cudaStreamSynchronize(c->st));
  // shifts that missed the tolerance: the plain FP64 path, one system each
  std::vector<long long> F;
  StreamIn sub;
  for (size_t k = 0; k < ne_c; ++k)
    if (sit[k] < 0) {
      F.push_back((long long)k);
      sub.E.push_back(E[k / n_cols]);
      sub.col.push_back(cols[k % n_cols]);
      sub.junc.push_back(0);
      sub.dep.push_back(-1);
      sub.bn2.push_back(0.0);
      sub.xo.push_back(full ? (long long)k * N : -1);
      sub.xfo.push_back(0);
    }
  std::string why;
  rsn_status worst = RSN_OK;
  if (!F.empty()) {
    StreamOut s2;
    if ((rs = run_stream(c, o, sub, full ? reinterpret_cast<double2*>(x_dev) : nullptr, nullptr, !full, 0, t_start,
                         s2)) != RSN_OK)
      return rs;
    for (size_t f = 0; f < F.size(); ++f) {
      sit[F[f]] = s2.status[f] == 0 ? -1000000 - s2.iters[f] : -std::max(1, s2.iters[f]);
      srel[F[f]] = s2.relres[f];
      if (!full)
        RSN_CUDA(c, cudaMemcpyAsync(q.t_all.as<double>() + F[f], q.out_t.as<double>() + f, sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->st));
    }
    c->st_fallback += (int64_t)F.size();
    worst = stream_status(s2, 0, (long long)F.size(), nullptr, nullptr, &why);
  }
  if (iters)
    for (size_t k = 0; k < ne_c; ++k)
      iters[k] = sit[k] >= 0 ? sit[k] : (sit[k] <= -1000000 ? -1000000 - sit[k] : sit[k]);
  if (relres)
    for (size_t k = 0; k < ne_c; ++k) relres[k] = srel[k];
  if (T) {
    RSN_CUDA(c, q.gr_cols.ensure(n_cols * sizeof(double)));
    RSN_CUDA(c, q.Td.ensure(n_e * sizeof(double)));
    std::vector<double> hgr(n_cols);
    for (int k = 0; k < n_cols; ++k) hgr[k] = c->gr[cols[k]];
    RSN_CUDA(c, cudaMemcpyAsync(q.gr_cols.p, hgr.data(), n_cols * sizeof(double), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, launch_t_final(n_e, n_cols, c->st, q.t_all.as<double>(), q.gr_cols.as<double>(), q.Td.as<double>()));
    RSN_CUDA(c, cudaMemcpyAsync(T, q.Td.p, n_e * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
  RSN_CUDA(c, cudaStreamSynchronize(c->st));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->t0, c->t1);
  c->st_ms = ms;
  if ((rs = leave(c)) != RSN_OK) return rs;
  if (worst != RSN_OK) RSN_FAIL(c, worst, "some shifted systems did not reach tol in the FP64 re-solve: %s", why.c_str());
  return RSN_OK;
}

extern "C" {

rsn_status rsn_solve_columns_shifted(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                     const rsn_solver_opts* o, void* x_dev, int32_t* iters, double* relres) {
  if (!c) return RSN_EINVAL;
  if ((long long)n_e * n_cols > 0 && !x_dev) RSN_FAIL(c, RSN_EINVAL, "x_dev is NULL");
  return shifted_impl(c, n_e, E, n_cols, cols, o, x_dev, iters, relres, nullptr);
}

rsn_status rsn_transmission_shifted(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                    const rsn_solver_opts* o, double* T, int32_t* iters) {
  if (!c) return RSN_EINVAL;
  if (n_e > 0 && !T) RSN_FAIL(c, RSN_EINVAL, "T is NULL");
  return shifted_impl(c, n_e, E, n_cols, cols, o, nullptr, iters, nullptr, T);
}

rsn_status rsn_transmission_keep(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                 const rsn_solver_opts* o, void* x_dev, double* T) {
  if (!c) return RSN_EINVAL;
  if (n_e > 0 && !T) RSN_FAIL(c, RSN_EINVAL, "T is NULL");
  if ((long long)n_e * n_cols > 0 && !x_dev) RSN_FAIL(c, RSN_EINVAL, "x_dev is NULL");
  return transmission_impl(c, n_e, E, n_cols, cols, o, nullptr, nullptr, 0, T, reinterpret_cast<double2*>(x_dev));
}

rsn_status rsn_transmission_vjp_reuse(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                      const rsn_solver_opts* o, const void* x_dev, const double* T_bar, double* dV,
                                      int dV_is_device) {
  if (!c) return RSN_EINVAL;
  if (!dV) RSN_FAIL(c, RSN_EINVAL, "dV is NULL");
  if ((long long)n_e * n_cols > 0 && !x_dev) RSN_FAIL(c, RSN_EINVAL, "x_dev is NULL");
  return transmission_impl(c, n_e, E, n_cols, cols, o, T_bar, dV, dV_is_device, nullptr, nullptr,
                           reinterpret_cast<const double2*>(x_dev));
}

}  // extern "C"

// Slot-pool description of several junctions for one precision: per-junction
// tilings for `nslots` slots, one launch configuration per operator kind in
// use (largest thread count, shared memory and tile count of its junctions).
// Register-kernel junctions must agree on points per thread (a template
// parameter); returns false if they do not.
static bool make_pool(rsn_ctx* const* ctxs, int K, bool fp32, int nslots, PoolSpec& pool,
                      std::vector<JuncDev>& js) {
  pool = PoolSpec();
  pool.K = K;
  pool.R = ctxs[0]->R;
  js.assign(2 * K, JuncDev{});
  int ppt_reg = 0, ppt_res = 0;
  for (int k = 0; k < K; ++k) {
    rsn_ctx* c = ctxs[k];
    const Tiling ti = choose_tiling(c, !fp32, OP_COCG, nslots), tr = choose_tiling(c, true, OP_RESID, nslots);
    const int kind = ti.plane ? kOpPlane : ti.pair ? kOpPair : ti.tma ? kOpTma : kOpReg;
    if (kind == kOpReg) {
      if (ppt_reg && ppt_reg != ti.ppt) return false;
      ppt_reg = ti.ppt;
    }
    if (ppt_res && ppt_res != tr.ppt) return false;
    ppt_res = tr.ppt;
    Tiling& L = pool.inner[kind];
    if (!pool.has[kind]) L = ti;
    pool.has[kind] = true;
    L.threads = std::max(L.threads, ti.threads);
    L.smem = std::max(L.smem, ti.smem);
    L.n = std::max(L.n, ti.n);
    L.big = L.big || ti.big;
    if (k == 0) pool.resid = tr;
    pool.resid.threads = std::max(pool.resid.threads, tr.threads);
    pool.resid.smem = std::max(pool.resid.smem, tr.smem);
    pool.resid.n = std::max(pool.resid.n, tr.n);
    pool.N = std::max(pool.N, c->N);
    pool.n_proj = std::max(pool.n_proj, c->n_proj);
    pool.n_groups = std::max(pool.n_groups, c->n_groups);
    pool.max_np = std::max(pool.max_np, c->max_np);
    pool.nB = std::max(pool.nB, c->jh.nB);
    pool.nS = std::max(pool.nS, c->jh.nS);
    pool.PA = std::max(pool.PA, std::max(ti.n + c->n_groups, tr.n));
    pool.PB = std::max(pool.PB, c->jh.nB);
    for (int h = 0; h < 2; ++h) {
      const Tiling& t = h == 0 ? ti : tr;
      JuncDev& J = js[h * K + k];
      J = c->jh;
      J.TY = t.TY;
      J.Lz = t.Lz;
      J.ytiles = t.ytiles;
      J.ztiles = t.ztiles;
      J.nA = t.n;
      J.nR = tr.n;
      J.kind = h == 0 ? kind : kOpReg;
    }
  }
  // the big point-pair variant serves every point-pair junction of the pool
  if (pool.has[kOpPair] && pool.inner[kOpPair].threads > kPairThreads) pool.inner[kOpPair].big = true;
  return true;
}

// rsn_batch_transmission on one slot pool: every (junction, energy, column)
// system of the batch waits in one queue, and each slot works on its system's
// junction, so uneven junctions share every launch.  The first context owns
// the pool (stream, slots, graphs).
static rsn_status batch_pool_impl(int K, rsn_ctx* const* ctxs, const int* n_e, const double* const* E,
                                  const int* n_cols, const int32_t* const* cols, const rsn_solver_opts* o,
                                  double* const* T, std::vector<rsn_status>& st) {
  rsn_ctx* c = ctxs[0];
  const bool fp32 = o->precision == RSN_MIXED;
  RSN_CUDA(c, cudaSetDevice(c->device));
  // order the pool's stream after every caller stream
  for (int k = 0; k < K; ++k) {
    RSN_CUDA(c, cudaEventRecord(ctxs[k]->ev_in, ctxs[k]->user_stream));
    RSN_CUDA(c, cudaStreamWaitEvent(c->st, ctxs[k]->ev_in, 0));
  }
  reset_stats(c);
  const auto t_start = std::chrono::steady_clock::now();
  RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
  StreamIn in;
  std::vector<long long> sys0(K + 1, 0), e0(K + 1, 0);
  std::vector<double> gr_all;
  for (int k = 0; k < K; ++k) {
    for (int e = 0; e < n_e[k]; ++e)
      for (int j = 0; j < n_cols[k]; ++j) {
        in.junc.push_back(k);
        in.E.push_back(E[k][e]);
        in.col.push_back(cols[k][j]);
        in.dep.push_back(-1);
        in.bn2.push_back(0.0);
        in.xo.push_back(-1);
        in.xfo.push_back(0);
      }
    sys0[k + 1] = (long long)in.E.size();
    e0[k + 1] = e0[k] + n_e[k];
    for (int j = 0; j < n_cols[k]; ++j) gr_all.push_back(ctxs[k]->gr[cols[k][j]]);
  }
  const long long nsys = sys0[K];
  CallBufs& q = c->cb;
  RSN_CUDA(c, q.gr_cols.ensure(std::max<size_t>(1, gr_all.size()) * sizeof(double)));
  RSN_CUDA(c, q.Td.ensure(std::max<long long>(1, e0[K]) * sizeof(double)));
  if (!gr_all.empty())
    RSN_CUDA(c, cudaMemcpyAsync(q.gr_cols.p, gr_all.data(), gr_all.size() * sizeof(double), cudaMemcpyHostToDevice,
                                c->st));
  std::vector<int> status(nsys, 0);
  std::vector<int> iters(nsys, 0);
  if (nsys > 0) {
    auto run = [&](const rsn_solver_opts* oo, const StreamIn& sin, StreamOut& so) -> rsn_status {
      const bool f32 = oo->precision == RSN_MIXED;
      // slots first (a pool of one slot size), then the tilings for that count
      PoolSpec probe;
      std::vector<JuncDev> js;
      probe.N = 0;
      for (int k = 0; k < K; ++k) probe.N = std::max(probe.N, ctxs[k]->N);
      const int S = choose_slots(c, oo, (long long)sin.E.size(), 0, 0, probe.N);
      rsn_solver_opts o2 = *oo;
      o2.rhs_block = S;
      PoolSpec pool;
      if (!make_pool(ctxs, K, f32, S, pool, js)) RSN_FAIL(c, RSN_EINVAL, "pool: junctions need different kernels");
      RSN_CUDA(c, c->pool_jd.ensure(js.size() * sizeof(JuncDev)));
      RSN_CUDA(c, cudaMemcpyAsync(c->pool_jd.p, js.data(), js.size() * sizeof(JuncDev), cudaMemcpyHostToDevice, c->st));
      RSN_CUDA(c, cudaStreamSynchronize(c->st));  // js lives on the host stack
      pool.ji = c->pool_jd.as<JuncDev>();
      pool.jr = c->pool_jd.as<JuncDev>() + K;
      // graphs captured for another configuration must not be replayed
      clear_graphs(c);
      c->ws.generation++;
      return run_stream(c, &o2, sin, nullptr, nullptr, true, 0, t_start, so, nullptr, &pool);
    };
    StreamOut so;
    rsn_status rs = run(o, in, so);
    if (rs != RSN_OK) return rs;
    RSN_CUDA(c, q.t_all.ensure(nsys * sizeof(double)));
    RSN_CUDA(c, cudaMemcpyAsync(q.t_all.p, q.out_t.p, nsys * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (fp32) {
      // systems whose FP32 recurrence stalled are solved again in FP64 (same pool)
      std::vector<long long> F;
      StreamIn sub;
      for (long long k = 0; k < nsys; ++k)
        if (so.status[k] != 0) {
          F.push_back(k);
          sub.push(in, (size_t)k);
          sub.bn2.back() = 0.0;
        }
      if (!F.empty()) {
        rsn_solver_opts o64;
        rsn_default_opts(RSN_FP64, &o64);
        o64.tol = o->tol;
        o64.tol_T = o->tol_T;
        o64.deadline_ms = o->deadline_ms;
        o64.use_graph = o->use_graph;
        o64.graph_iters = o->graph_iters;
        StreamOut s2;
        if ((rs = run(&o64, sub, s2)) != RSN_OK) return rs;
        for (size_t f = 0; f < F.size(); ++f) {
          so.status[F[f]] = s2.status[f];
          so.iters[F[f]] += s2.iters[f];
          so.relres[F[f]] = s2.relres[f];
          RSN_CUDA(c, cudaMemcpyAsync(q.t_all.as<double>() + F[f], q.out_t.as<double>() + f, sizeof(double),
                                      cudaMemcpyDeviceToDevice, c->st));
        }
        c->st_fallback += (int64_t)F.size();
      }
    }
    for (int k = 0; k < K; ++k) {
      if (n_e[k] == 0) continue;
      if (n_cols[k] == 0) {
        RSN_CUDA(c, cudaMemsetAsync(q.Td.as<double>() + e0[k], 0, n_e[k] * sizeof(double), c->st));
        continue;
      }
      long long c0 = 0;
      for (int l = 0; l < k; ++l) c0 += n_cols[l];
      RSN_CUDA(c, launch_t_final(n_e[k], n_cols[k], c->st, q.t_all.as<double>() + sys0[k],
                                 q.gr_cols.as<double>() + c0, q.Td.as<double>() + e0[k]));
    }
    for (long long k = 0; k < nsys; ++k) status[k] = so.status[k], iters[k] = so.iters[k];
    for (int k = 0; k < K; ++k) {
      std::string why;
      StreamOut part;
      part.status.assign(so.status.begin() + sys0[k], so.status.begin() + sys0[k + 1]);
      part.iters.assign(so.iters.begin() + sys0[k], so.iters.begin() + sys0[k + 1]);
      part.relres.assign(so.relres.begin() + sys0[k], so.relres.begin() + sys0[k + 1]);
      part.timeout = so.timeout;
      const rsn_status ks = stream_status(part, 0, sys0[k + 1] - sys0[k], nullptr, nullptr, &why);
      if (ks != RSN_OK) {
        st[k] = ks;
        char buf[600];
        snprintf(buf, sizeof(buf), "some systems did not reach tol: %s", why.c_str());
        ctxs[k]->err = buf;
      }
    }
  }
  RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
  for (int k = 0; k < K; ++k)
    if (n_e[k] > 0)
      RSN_CUDA(c, cudaMemcpyAsync(T[k], q.Td.as<double>() + e0[k], n_e[k] * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->st));
  RSN_CUDA(c, cudaStreamSynchronize(c->st));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->t0, c->t1);
  c->st_ms = ms;
  clear_graphs(c);
  c->ws.generation++;
  // every caller stream waits for the pool's work
  RSN_CUDA(c, cudaEventRecord(c->ev_out, c->st));
  for (int k = 0; k < K; ++k) RSN_CUDA(c, cudaStreamWaitEvent(ctxs[k]->user_stream, c->ev_out, 0));
  return RSN_OK;
}

extern "C" {

rsn_status rsn_batch_transmission(int n_ctx, rsn_ctx* const* ctxs, const int* n_e, const double* const* E,
                                  const int* n_cols, const int32_t* const* cols, const rsn_solver_opts* opts,
                                  double* const* T, rsn_status* status) {
  if (n_ctx < 0) return RSN_EINVAL;
  if (n_ctx == 0) return RSN_OK;
  if (!ctxs || !n_e || !E || !n_cols || !cols || !T) return RSN_EINVAL;
  for (int k = 0; k < n_ctx; ++k) {
    if (!ctxs[k]) return RSN_EINVAL;
    for (int l = 0; l < k; ++l)
      if (ctxs[l] == ctxs[k]) RSN_FAIL(ctxs[k], RSN_EINVAL, "context %d repeats context %d", k, l);
  }
  rsn_solver_opts base;
  if (opts) base = *opts;
  else rsn_default_opts(RSN_MIXED, &base);
  // one slot pool when every junction is on the same device with the same FD
  // order and no explicit slot count was asked for
  bool pooled = n_ctx > 1 && base.rhs_block <= 0;
  for (int k = 0; k < n_ctx && pooled; ++k) pooled = ctxs[k]->device == ctxs[0]->device && ctxs[k]->R == ctxs[0]->R;
  if (pooled) {
    std::vector<rsn_status> st(n_ctx, RSN_OK);
    for (int k = 0; k < n_ctx; ++k) {
      rsn_ctx* c = ctxs[k];
      rsn_status rs = RSN_OK;
      if (n_e[k] > 0 && !T[k]) {
        c->err = "T is NULL";
        rs = RSN_EINVAL;
      }
      if (rs == RSN_OK) rs = commit_setup(c);
      if (rs == RSN_OK) rs = check_solve_args(c, n_e[k], E[k], n_cols[k], cols[k], &base);
      st[k] = rs;
    }
    int bad = -1;
    for (int k = 0; k < n_ctx && bad < 0; ++k)
      if (st[k] != RSN_OK) bad = k;
    if (bad >= 0) {
      // the pool runs all junctions or none
      for (int k = 0; k < n_ctx; ++k)
        if (st[k] == RSN_OK) {
          st[k] = RSN_EINVAL;
          ctxs[k]->err = "rsn_batch_transmission: not run, the arguments of junction " + std::to_string(bad) +
                         " were refused";
        }
    } else {
      const rsn_status rs = batch_pool_impl(n_ctx, ctxs, n_e, E, n_cols, cols, &base, T, st);
      if (rs != RSN_OK)
        for (int k = 0; k < n_ctx; ++k)
          if (st[k] == RSN_OK) {
            st[k] = rs;
            if (k) ctxs[k]->err = "rsn_batch_transmission: the slot pool failed: " + ctxs[0]->err;
          }
    }
    rsn_status worst = RSN_OK;
    for (int k = 0; k < n_ctx; ++k) {
      if (status) status[k] = st[k];
      if (worst == RSN_OK && st[k] != RSN_OK) worst = st[k];
    }
    return worst;
  }
  // per-context options: without an explicit slot count, each context's pool
  // is capped by its share of the free memory of its device
  std::vector<rsn_solver_opts> ok(n_ctx, base);
  std::map<int, int> per_dev;
  for (int k = 0; k < n_ctx; ++k) per_dev[ctxs[k]->device]++;
  std::map<int, size_t> free_dev;
  for (auto& d : per_dev) {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(d.first) == cudaSuccess && cudaMemGetInfo(&fr, &tot) == cudaSuccess) free_dev[d.first] = fr;
    else free_dev[d.first] = 0;
  }
  if (base.rhs_block <= 0) {
    for (int k = 0; k < n_ctx; ++k) {
      rsn_ctx* c = ctxs[k];
      const double share = 0.6 * (double)free_dev[c->device] / per_dev[c->device];
      const long long cap = (long long)(share / (double)slot_bytes(c, base.precision == RSN_MIXED));
      ok[k].rhs_block = (int)std::max<long long>(1, std::min<long long>(cap, 2048));
    }
  }
  // order each context's work after its caller's stream once, up front, and
  // let the per-call stream handshake use the context's own stream: contexts
  // that share a caller stream (one framework stream) then do not wait for
  // one another; the caller's streams wait for the results at the end
  std::vector<cudaStream_t> user(n_ctx);
  for (int k = 0; k < n_ctx; ++k) {
    rsn_ctx* c = ctxs[k];
    RSN_CUDA(c, cudaSetDevice(c->device));
    RSN_CUDA(c, cudaEventRecord(c->ev_in, c->user_stream));
    RSN_CUDA(c, cudaStreamWaitEvent(c->st, c->ev_in, 0));
  }
  for (int k = 0; k < n_ctx; ++k) {
    user[k] = ctxs[k]->user_stream;
    ctxs[k]->user_stream = ctxs[k]->st;
  }
  std::vector<rsn_status> st(n_ctx, RSN_OK);
  std::vector<std::thread> th;
  th.reserve(n_ctx);
  for (int k = 0; k < n_ctx; ++k)
    th.emplace_back([&, k]() {
      cudaSetDevice(ctxs[k]->device);  // a new host thread starts on device 0
      if (n_e[k] > 0 && !T[k]) {
        st[k] = RSN_EINVAL;
        ctxs[k]->err = "T is NULL";
        return;
      }
      st[k] = transmission_impl(ctxs[k], n_e[k], E[k], n_cols[k], cols[k], &ok[k], nullptr, nullptr, 0, T[k]);
    });
  for (auto& t : th) t.join();
  for (int k = 0; k < n_ctx; ++k) {
    rsn_ctx* c = ctxs[k];
    c->user_stream = user[k];
    if (cudaSetDevice(c->device) != cudaSuccess || cudaEventRecord(c->ev_out, c->st) != cudaSuccess ||
        cudaStreamWaitEvent(c->user_stream, c->ev_out, 0) != cudaSuccess) {
      if (st[k] == RSN_OK) {
        st[k] = RSN_ECUDA;
        c->err = "rsn_batch_transmission: ordering the caller's stream after the context failed";
      }
    }
  }
  rsn_status worst = RSN_OK;
  for (int k = 0; k < n_ctx; ++k) {
    if (status) status[k] = st[k];
    if (worst == RSN_OK && st[k] != RSN_OK) worst = st[k];
  }
  return worst;
}

// One kernel of the COCG iteration in isolation: every slot ACTIVE with a
// synthetic, finite state; `reps` back-to-back launches timed with CUDA events.
static rsn_status bench_kernel_impl(rsn_ctx* c, int precision, int kind, int S, int reps, double* ms_out,
                                    double* bytes_out, int active = -1) {
  if (active < 0 || active > S) active = S;  // the first `active` slots work, the rest are free
  const bool fp32 = precision == RSN_MIXED;
  rsn_status rs = ensure_ws(c, fp32, S);
  if (rs != RSN_OK) return rs;
  Workspace& w = c->ws;
  cudaStream_t st = c->st;
  const long long N = c->N;
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  const size_t vb = (size_t)S * N;
  for (DevBuf* v : {&w.r, &w.p0, &w.p1, &w.q, &w.d}) RSN_CUDA(c, cudaMemsetAsync(v->p, 0x3c, vb * el, st));
  RSN_CUDA(c, cudaMemsetAsync(w.Xslot.p, 0x3c, vb * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.rho.p, 0x3f, (size_t)S * w.PB * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.rho_cur.p, 0x3f, S * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.sigma.p, 0, S * sizeof(double), st));
  RSN_CUDA(c, cudaMemsetAsync(w.beta_cur.p, 0x3f, S * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.nrm.p, 0x3f, (size_t)S * w.PB * sizeof(double), st));
  RSN_CUDA(c, cudaMemsetAsync(w.mu.p, 0x3f, (size_t)S * w.PA * sizeof(double2), st));
  const size_t npj = std::max(1, c->n_proj);
  RSN_CUDA(c, cudaMemsetAsync(w.c_r.p, 0, (size_t)S * npj * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.c_p.p, 0, 2 * (size_t)S * npj * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.c_x.p, 0, (size_t)S * npj * sizeof(double2), st));
  std::vector<int> hstate(S, kind == 2 ? SL_CHECK : SL_ACTIVE), hone(S, 1), hzero(S, 0), hcol(S, 0);
  for (int k = active; k < S; ++k) hstate[k] = SL_FREE;
  std::vector<double> hE(S, 0.2);
  std::vector<long long> hvo(S);
  for (int s = 0; s < S; ++s) hvo[s] = (long long)s * N;
  RSN_CUDA(c, cudaMemcpyAsync(w.state.p, hstate.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.iters.p, hone.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.junc.p, hzero.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.col.p, hcol.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.E.p, hE.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.xo.p, hvo.data(), S * sizeof(long long), cudaMemcpyHostToDevice, st));
  rsn_solver_opts o;
  rsn_default_opts(precision, &o);
  BatchDev b = slot_batch(c, S, &o);
  RSN_CUDA(c, cudaMemcpyAsync(c->bd.p, &b, sizeof(b), cudaMemcpyHostToDevice, st));
  const BatchDev* bdev = c->bd.as<BatchDev>();
  LaunchCfg cfg;
  if ((rs = make_cfg(c, fp32, S, cfg)) != RSN_OK) return rs;
  auto launch = [&]() -> cudaError_t {
    if (kind == 0) return launch_inner(c, cfg.inner, OP_COCG, fp32, S, st, cfg.jt_inner, bdev, nullptr, nullptr, nullptr);
    if (kind == 1) return launch_cocg_update(fp32, S, c->jh.nB, b.ce_stride, st, cfg.jt_inner, bdev);
    return launch_op(OP_RESID, fp32, c->R, cfg.resid.ppt, dim3(cfg.resid.n, S), cfg.resid.threads, cfg.resid.smem,
                     st, cfg.jt_resid, bdev, nullptr, nullptr, nullptr);
  };
  RSN_CUDA(c, launch_list(st, bdev));  // every slot, for the true-residual kernel
  for (int i = 0; i < 2; ++i) RSN_CUDA(c, launch());
  RSN_CUDA(c, cudaEventRecord(c->t0, st));
  for (int i = 0; i < reps; ++i) RSN_CUDA(c, launch());
  RSN_CUDA(c, cudaEventRecord(c->t1, st));
  RSN_CUDA(c, cudaEventSynchronize(c->t1));
  float ms = 0.f;
  RSN_CUDA(c, cudaEventElapsedTime(&ms, c->t0, c->t1));
  if (ms_out) *ms_out = ms / reps;
  const double v = (double)N * active;
  if (bytes_out)
    *bytes_out = kind == 0 ? 4.0 * el * v : kind == 1 ? 6.0 * el * v : (sizeof(double2) + 2.0 * el) * v;
  return RSN_OK;
}

rsn_status rsn_bench_kernel(rsn_ctx* c, int precision, int kind, int nslots, int reps, double* ms_per_launch,
                            double* bytes_per_launch) {
  if (!c) return RSN_EINVAL;
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((precision != RSN_FP64 && precision != RSN_MIXED) || kind < 0 || kind > 2 || nslots < 1 || reps < 1)
    RSN_FAIL(c, RSN_EINVAL, "bad benchmark arguments");
  if ((rs = enter(c)) != RSN_OK) return rs;
  if ((rs = bench_kernel_impl(c, precision, kind, nslots, reps, ms_per_launch, bytes_per_launch)) != RSN_OK)
    return rs;
  return leave(c);
}

// Search the operator kernel's tiling for this grid, precision and slot count:
// plane-streaming kernel with several z-chunk lengths, and the register-prefetch
// kernel over (TY, ppt, Lz).  The fastest is kept as the context's tiling.
rsn_status rsn_autotune(rsn_ctx* c, int precision, int nslots, int* TY, int* Lz, int* ppt, int* tma,
                        double* best_gbs) {
  if (!c) return RSN_EINVAL;
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((precision != RSN_FP64 && precision != RSN_MIXED) || nslots < 1) RSN_FAIL(c, RSN_EINVAL, "bad arguments");
  if ((rs = enter(c)) != RSN_OK) return rs;
  const bool fp32 = precision == RSN_MIXED;
  struct Cand { int TY, Lz, ppt, notma; };
  std::vector<Cand> cands;
  std::vector<int> lzs;
  for (int zt : {1, 2, 3, 4, 6, 8}) {
    const int lz = (c->nz + zt - 1) / zt;
    if (lz >= 2 * c->R + 2 || zt == 1) lzs.push_back(lz);
  }
  for (int lz : lzs) cands.push_back({0, lz, 0, -2});  // FP32 point-pair kernel where it applies
  for (int lz : lzs) cands.push_back({0, lz, 0, -3});  // FP32 plane kernel where it applies
  for (int lz : lzs) cands.push_back({0, lz, 0, -1});  // whole-plane bulk-copy kernel
  for (int p = 1; p <= 4; ++p)
    for (int ty : {c->ny, (c->ny + 1) / 2, (c->ny + 2) / 3})
      for (int lz : lzs) {
        const int thr = (c->nx * ty + p - 1) / p;
        if (thr < 32 || thr > 256) continue;
        cands.push_back({ty, lz, p, 1});
      }
  const int save[4] = {c->tile_override[0], c->tile_override[1], c->tile_override[2], c->tile_override[3]};
  double best = -1.0;
  Cand bestc = {0, 0, 0, 0};
  // objective: the launch time with every slot active plus the time with a
  // quarter of them active (the tail of a stream, where long z chunks leave
  // SMs idle); reported: the algorithmic GB/s with every slot active
  double best_score = 1e300;
  for (const Cand& k : cands) {
    c->tile_override[0] = k.TY;
    c->tile_override[1] = k.Lz;
    c->tile_override[2] = k.ppt;
    c->tile_override[3] = k.notma;
    c->ws.slots = 0;
    double ms = 0, by = 0, ms_q = 0, by_q = 0;
    rs = bench_kernel_impl(c, precision, 0, nslots, 5, &ms, &by);
    if (rs != RSN_OK) continue;  // e.g. a shared-memory size this tile cannot have
    rs = bench_kernel_impl(c, precision, 0, nslots, 5, &ms_q, &by_q, std::max(1, nslots / 4));
    if (rs != RSN_OK) continue;
    const double score = ms + ms_q;
    if (score < best_score) {
      best_score = score;
      best = by / (ms * 1e6);
      bestc = k;
    }
  }
  if (best < 0) {
    for (int i = 0; i < 4; ++i) c->tile_override[i] = save[i];
    RSN_FAIL(c, RSN_ECUDA, "no tiling candidate ran");
  }
  c->tile_override[0] = bestc.TY;
  c->tile_override[1] = bestc.Lz;
  c->tile_override[2] = bestc.ppt;
  c->tile_override[3] = bestc.notma;
  c->ws.slots = 0;
  clear_graphs(c);
  c->ws.generation++;
  c->err.clear();
  if (TY) *TY = bestc.TY;
  if (Lz) *Lz = bestc.Lz;
  if (ppt) *ppt = bestc.ppt;
  if (tma) {
    const Tiling tb = choose_tiling(c, !fp32, OP_COCG, nslots);
    *tma = tb.plane ? 3 : tb.pair ? 2 : tb.tma ? 1 : 0;
  }
  if (best_gbs) *best_gbs = best;
  (void)fp32;
  return leave(c);
}

rsn_status rsn_landauer_current(rsn_ctx* c, int n_e, const double* E, const double* T, int n_v, const double* V,
                                double E_F, double kT, double* I) {
  if (!c) return RSN_EINVAL;
  if (n_e < 0 || n_v < 0 || (n_e > 0 && (!E || !T)) || (n_v > 0 && (!V || !I)))
    RSN_FAIL(c, RSN_EINVAL, "bad arguments");
  if (!(kT >= 0.0) || !std::isfinite(kT) || !std::isfinite(E_F)) RSN_FAIL(c, RSN_EINVAL, "kT must be >= 0, E_F finite");
  for (int e = 0; e < n_e; ++e) {
    if (!std::isfinite(E[e]) || !std::isfinite(T[e])) RSN_FAIL(c, RSN_EINVAL, "E[%d] or T[%d] is not finite", e, e);
    if (e > 0 && !(E[e] > E[e - 1])) RSN_FAIL(c, RSN_EINVAL, "energies must be strictly ascending (index %d)", e);
  }
  for (int k = 0; k < n_v; ++k)
    if (!std::isfinite(V[k])) RSN_FAIL(c, RSN_EINVAL, "V[%d] is not finite", k);
  if (n_v == 0) return RSN_OK;
  if (n_e < 2) {
    for (int k = 0; k < n_v; ++k) I[k] = 0.0;
    return RSN_OK;
  }
  rsn_status rs = enter(c);
  if (rs != RSN_OK) return rs;
  CallBufs& q = c->cb;
  auto body = [&]() -> rsn_status {
    RSN_CUDA(c, q.lE.ensure(n_e * sizeof(double)));
    RSN_CUDA(c, q.lT.ensure(n_e * sizeof(double)));
    RSN_CUDA(c, q.lV.ensure(n_v * sizeof(double)));
    RSN_CUDA(c, q.lI.ensure(n_v * sizeof(double)));
    RSN_CUDA(c, cudaMemcpyAsync(q.lE.p, E, n_e * sizeof(double), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, cudaMemcpyAsync(q.lT.p, T, n_e * sizeof(double), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, cudaMemcpyAsync(q.lV.p, V, n_v * sizeof(double), cudaMemcpyHostToDevice, c->st));
    RSN_CUDA(c, launch_landauer(n_e, q.lE.as<double>(), q.lT.as<double>(), n_v, q.lV.as<double>(), E_F, kT,
                                q.lI.as<double>(), c->st));
    RSN_CUDA(c, cudaMemcpyAsync(I, q.lI.p, n_v * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    RSN_CUDA(c, cudaStreamSynchronize(c->st));
    return RSN_OK;
  };
  rs = body();
  const rsn_status rl = leave(c);
  return rs != RSN_OK ? rs : rl;
}

// Tiling override used by the autotuner and the tests: TY, Lz, ppt (0 = auto).
rsn_status rsn_set_tiling(rsn_ctx* c, int TY, int Lz, int ppt) {
  if (!c) return RSN_EINVAL;
  if (TY < 0 || Lz < 0 || ppt < -3 || ppt > 4) RSN_FAIL(c, RSN_EINVAL, "bad tiling override");
  c->tile_override[0] = TY;
  c->tile_override[1] = Lz;
  c->tile_override[2] = ppt > 0 ? ppt : 0;
  c->tile_override[3] = ppt < 0 ? ppt : 0;
  clear_graphs(c);
  c->ws.generation++;
  c->ws.slots = 0;  // partial strides may change
  return RSN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free operator application.
//
// Callers that cannot allocate device memory during a call -- code running
// where cudaMalloc is forbidden or unsafe (inside a pre-sized memory pool, a
// real-time loop, or a host framework that owns every allocation) -- can apply
// A(E) through rsn_apply_noalloc.  Its per-call scratch (the launch
// descriptor, the per-vector energy / offset / junction tables and the
// projector coefficients) lives in the fixed array below instead of library
// allocations.  Every device that loads the library holds this array until the
// process exits.  All calls share it and it keeps the last call's contents;
// every field a call reads is rewritten by that call before use, so nothing
// needs clearing, but calls that overlap on the GPU (other streams or host
// threads) race on it.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB per device
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// per-vector offsets and junction ids of the scratch tables (filled on the device)
__global__ void noalloc_tables_kernel(int n, long long N, long long* voff, int* junc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    voff[s] = (long long)s * N;
    junc[s] = 0;
  }
}

// The work of one allocation-free call, between enter() and leave().
static rsn_status apply_noalloc_impl(rsn_ctx* c, int precision, int n_rhs, const double* E, const void* x_dev,
                                     void* y_dev, unsigned char* base, size_t o_E, size_t o_voff, size_t o_junc,
                                     size_t o_c) {
  const bool fp32 = precision == RSN_MIXED;
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.nslots = n_rhs;
  b.E = reinterpret_cast<double*>(base + o_E);
  b.voff = reinterpret_cast<long long*>(base + o_voff);
  b.junc = reinterpret_cast<int*>(base + o_junc);
  b.pstride = c->n_proj;
  void* cbuf = base + o_c;
  const BatchDev* bdev = reinterpret_cast<const BatchDev*>(base);
  RSN_CUDA(c, cudaMemcpyAsync(base, &b, sizeof(b), cudaMemcpyHostToDevice, c->st));
  RSN_CUDA(c, cudaMemcpyAsync(b.E, E, n_rhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
  noalloc_tables_kernel<<<(n_rhs + 255) / 256, 256, 0, c->st>>>(n_rhs, c->N, b.voff, b.junc);
  RSN_CUDA(c, cudaGetLastError());
  // bulk-copy kernels need 16-byte aligned vectors; otherwise a register tiling
  const bool aligned = (reinterpret_cast<uintptr_t>(x_dev) % 16) == 0 && (reinterpret_cast<uintptr_t>(y_dev) % 16) == 0;
  const Tiling t = choose_tiling(c, !fp32, OP_APPLY, n_rhs, aligned);
  LaunchCfg cfg;
  rsn_status rs = make_cfg(c, t, choose_tiling(c, true, OP_RESID, n_rhs), cfg);
  if (rs != RSN_OK) return rs;
  if (c->n_proj > 0)
    RSN_CUDA(c, launch_project(2, fp32, n_rhs, c->n_groups, c->max_np, c->st, cfg.jt_inner, bdev, x_dev, cbuf));
  RSN_CUDA(c, launch_inner(c, t, OP_APPLY, fp32, n_rhs, c->st, cfg.jt_inner, bdev, x_dev, y_dev, cbuf));
  return RSN_OK;
}

extern "C" rsn_status rsn_apply_noalloc(rsn_ctx* c, int precision, int n_rhs, const double* E, const void* x_dev,
                                        void* y_dev) {
  static std::mutex mu;
  static void* scratch_addr[kNoAllocMaxDevices] = {nullptr};
  if (!c) return RSN_EINVAL;
  if (n_rhs < 0 || (n_rhs > 0 && (!E || !x_dev || !y_dev))) RSN_FAIL(c, RSN_EINVAL, "bad arguments");
  if (precision != RSN_FP64 && precision != RSN_MIXED) RSN_FAIL(c, RSN_EINVAL, "bad precision");
  if (!c->has_grid || !c->has_v || !c->has_cap || c->dirty || !c->jd.p)
    RSN_FAIL(c, RSN_ESTATE,
             "rsn_apply_noalloc: the operator data is not on the device yet; an allocating call "
             "(e.g. rsn_apply) after the last setter uploads it");
  if (n_rhs == 0) return RSN_OK;
  // scratch layout: [BatchDev | E | voff | junc | projector coefficients]
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_E = up(sizeof(BatchDev));
  const size_t o_voff = up(o_E + (size_t)n_rhs * sizeof(double));
  const size_t o_junc = up(o_voff + (size_t)n_rhs * sizeof(long long));
  const size_t o_c = up(o_junc + (size_t)n_rhs * sizeof(int));
  const size_t need = o_c + (size_t)n_rhs * std::max(1, c->n_proj) * sizeof(double2);
  if (need > kNoAllocScratchBytes)
    RSN_FAIL(c, RSN_EINVAL,
             "rsn_apply_noalloc: %d vectors with %d projectors need %zu bytes of scratch, more than the %zu-byte "
             "fixed array; split the call",
             n_rhs, c->n_proj, need, kNoAllocScratchBytes);
  if (n_rhs > kMaxApplyRhs)
    RSN_FAIL(c, RSN_EINVAL, "rsn_apply_noalloc: n_rhs = %d exceeds %d vectors per call; split the call", n_rhs,
             kMaxApplyRhs);
  if (c->device < 0 || c->device >= kNoAllocMaxDevices) RSN_FAIL(c, RSN_EINVAL, "device index too large");
  rsn_status rs = enter(c);  // makes the context's device current
  if (rs != RSN_OK) return rs;
  unsigned char* base = nullptr;
  {
    // first call on a device: host code needs the device address of the array
    std::lock_guard<std::mutex> lock(mu);
    if (!scratch_addr[c->device]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e == cudaSuccess) scratch_addr[c->device] = p;
      else c->err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    }
    base = static_cast<unsigned char*>(scratch_addr[c->device]);
  }
  rs = base ? apply_noalloc_impl(c, precision, n_rhs, E, x_dev, y_dev, base, o_E, o_voff, o_junc, o_c) : RSN_ECUDA;
  // the caller's stream is ordered after whatever was queued, also on failure
  const rsn_status rl = leave(c);
  return rs != RSN_OK ? rs : rl;
}
