// C-ABI entry points, device-side setup of the operator data, and the host
// driver of the batched COCG solve with FP64 iterative refinement.
//
// Solve schedule for one batch of systems A(E_s) x_s = b_s (all in one stream):
//   repeat (refinement sweep):
//     [project x64 + d]  -> c_x                    (projector gathers, FP64)
//     op(RESID)          -> r = b - A(x64 + d), ||r||^2, r^T r   (FP64 arithmetic)
//     x_update           -> x64 += d, d = 0
//     outer_book         -> converged?  else restart the inner solve on r
//     [project r]        -> c_r
//     repeat (captured CUDA graph of `graph_iters` COCG iterations):
//        op(COCG)    p = r + beta p ; q = A p ; partial mu = p^T q
//        cocg_update alpha = rho/mu ; r -= alpha q ; d += alpha p ; partial rho, ||r||^2
//        [project r] -> c_r for the next iteration
//        inner_book  iteration counts, convergence, breakdown, active count
//     until no inner solve is active
//   until no system is active
// The host reads one integer per graph replay; everything else stays on the GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
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
};

struct Workspace {
  int slots = 0;
  bool fp32 = false;
  bool adjoint = false;
  long long N = 0;
  int PA = 0, PB = 0, n_proj = 0;
  DevBuf X0, X1, r, p0, p1, q, d;
  DevBuf junc, E, col, voff, iters, done, outer_done, total_iters, n_outer, status, breakdowns;
  DevBuf bnorm2, tol2, relres, out_index, wt;
  DevBuf rho0, nrm0, rho, nrm, mu, c_r, c_p, c_x, n_active;
  int generation = 0;
};

struct GraphKey {
  int fp32, slots, iters, generation, proj;
  bool operator<(const GraphKey& o) const {
    return std::tie(fp32, slots, iters, generation, proj) < std::tie(o.fp32, o.slots, o.iters, o.generation, o.proj);
  }
};

}  // namespace

struct rsn_ctx {
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
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
  DevBuf dg64, dg32, gld, L_idx, L_gam, inv_ptr, inv_proj, inv_val64, inv_val32;
  DevBuf grp_ptr, grp_p0, grp_np, grp_voff, grp_idx, grp_val64, grp_val32, ekb;
  int n_groups = 0, nL = 0;
  JuncDev jh{};
  DevBuf jd;  // device JuncDev (one per launch configuration, uploaded before a batch)

  Workspace ws;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  int* n_active_host = nullptr;  // pinned

  // stats of the last solve
  int64_t st_iters = 0, st_sweeps = 0, st_launches = 0;
  double st_ms = 0.0;
  int tile_override[4] = {0, 0, 0, 0};  // TY, Lz, ppt, unused (autotuner / tests)
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
static Tiling choose_tiling(const rsn_ctx* c, bool compute64, int mode, int nslots) {
  Tiling t;
  const int nx = c->nx, ny = c->ny, nz = c->nz, R = c->R;
  const int qregs = (2 * R + 1) * (compute64 ? 4 : 2);
  int ppt_max = std::max(1, std::min(4, 64 / qregs));
  int TY = ny;
  if ((long long)nx * ny > 512LL * ppt_max) {
    const int tymax = std::max(1, (512 * ppt_max) / nx);
    const int yt = (ny + tymax - 1) / tymax;
    TY = (ny + yt - 1) / yt;
  }
  int ppt = std::min(ppt_max, std::max(1, (nx * TY + 383) / 384));
  if (c->tile_override[0] > 0) TY = std::min(ny, c->tile_override[0]);
  if (c->tile_override[2] > 0) ppt = std::min(4, c->tile_override[2]);
  int threads = (nx * TY + ppt - 1) / ppt;
  threads = ((threads + 31) / 32) * 32;
  while (threads > 512 && ppt < 4) {
    ++ppt;
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
  t.Lz = (nz + zt - 1) / zt;
  t.ztiles = (nz + t.Lz - 1) / t.Lz;
  t.n = t.ytiles * t.ztiles;
  t.smem = op_smem_bytes(!compute64, mode, R, TY, nx, c->n_proj);
  return t;
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
    dgf[i] = make_float2((float)dg[i].x, (float)dg[i].y);
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
    for (int k = 0; k < np; ++k)
      for (int64_t e = c->poff[k]; e < c->poff[k + 1]; ++e) cnt[c->pidx[e] + 1]++;
  }
  c->n_groups = (int)gp0.size();
  for (long long i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  const size_t nnz = (size_t)cnt[N];
  std::vector<int> iproj(std::max<size_t>(1, nnz)), fill(cnt.begin(), cnt.end() - 1);
  std::vector<double> ival(std::max<size_t>(1, nnz));
  for (int k = 0; k < np; ++k)
    for (int64_t e = c->poff[k]; e < c->poff[k + 1]; ++e) {
      const int i = c->pidx[e];
      iproj[fill[i]] = k;
      ival[fill[i]] = c->pval[e];
      fill[i]++;
    }
  std::vector<float> ivalf(ival.begin(), ival.end()), gvalf(gval.begin(), gval.end());
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = b.ensure(std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    if (bytes) return cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice);
    return cudaSuccess;
  };
  RSN_CUDA(c, up(c->inv_ptr, cnt.data(), (N + 1) * sizeof(int)));
  RSN_CUDA(c, up(c->inv_proj, iproj.data(), nnz * sizeof(int)));
  RSN_CUDA(c, up(c->inv_val64, ival.data(), nnz * sizeof(double)));
  RSN_CUDA(c, up(c->inv_val32, ivalf.data(), nnz * sizeof(float)));
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
  J.inv_proj = c->inv_proj.as<int>();
  J.inv_val64 = c->inv_val64.as<double>();
  J.inv_val32 = c->inv_val32.as<float>();
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

static rsn_status make_cfg(rsn_ctx* c, bool fp32, int nslots, LaunchCfg& cfg) {
  cfg.inner = choose_tiling(c, !fp32, OP_COCG, nslots);
  cfg.resid = choose_tiling(c, true, OP_RESID, nslots);
  JuncDev js[2] = {c->jh, c->jh};
  for (int k = 0; k < 2; ++k) {
    const Tiling& t = k == 0 ? cfg.inner : cfg.resid;
    js[k].TY = t.TY;
    js[k].Lz = t.Lz;
    js[k].ytiles = t.ytiles;
    js[k].ztiles = t.ztiles;
    js[k].nA = t.n;
    js[k].nR = cfg.resid.n;
  }
  RSN_CUDA(c, cudaMemcpyAsync(c->jd.p, js, 2 * sizeof(JuncDev), cudaMemcpyHostToDevice, c->st));
  cfg.jt_inner = c->jd.as<JuncDev>();
  cfg.jt_resid = c->jd.as<JuncDev>() + 1;
  return RSN_OK;
}

extern "C" {

void rsn_default_opts(int precision, rsn_solver_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = precision == RSN_MIXED ? RSN_MIXED : RSN_FP64;
  if (o->precision == RSN_MIXED) {
    o->tol = 1e-10;
    o->tol_inner = 1e-5;
  } else {
    o->tol = 1e-13;
    o->tol_inner = 1e-11;
  }
  o->max_iter = 4000;
  o->max_outer = 8;
  o->deadline_ms = 0.0;
  o->rhs_block = 0;
  o->use_graph = 1;
  o->graph_iters = 16;
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
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&c->t0) != cudaSuccess || cudaEventCreate(&c->t1) != cudaSuccess ||
      cudaMallocHost(&c->n_active_host, 4 * sizeof(int)) != cudaSuccess) {
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
  clear_graphs(c);
  if (c->n_active_host) cudaFreeHost(c->n_active_host);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->t0) cudaEventDestroy(c->t0);
  if (c->t1) cudaEventDestroy(c->t1);
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

rsn_status rsn_last_stats(const rsn_ctx* c, int64_t* it, int64_t* sw, int64_t* la, double* ms) {
  if (!c) return RSN_EINVAL;
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
// workspace
// ---------------------------------------------------------------------------
static size_t per_slot_bytes(const rsn_ctx* c, bool fp32, bool adjoint) {
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  return (size_t)c->N * (sizeof(double2) * (adjoint ? 2 : 1) + 5 * el) + 4096;
}

static int choose_slots(rsn_ctx* c, const rsn_solver_opts* o, bool adjoint, long long total) {
  if (o->rhs_block > 0) return (int)std::min<long long>(o->rhs_block, total);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const size_t per = per_slot_bytes(c, o->precision == RSN_MIXED, adjoint);
  long long cap = (long long)(0.5 * (double)fr / (double)per);
  cap = std::max<long long>(1, std::min<long long>(cap, 16384));
  return (int)std::min<long long>(cap, total);
}

static rsn_status ensure_ws(rsn_ctx* c, bool fp32, bool adjoint, int slots, bool own_x0) {
  Workspace& w = c->ws;
  const long long N = c->N;
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  const Tiling ti = choose_tiling(c, !fp32, OP_COCG, slots), tr = choose_tiling(c, true, OP_RESID, slots);
  const int PA = std::max(ti.n, tr.n), PB = c->jh.nB;
  const bool same = w.slots == slots && w.fp32 == fp32 && w.N == N && w.PA == PA && w.PB == PB &&
                    w.n_proj == c->n_proj && (!adjoint || w.adjoint);
  if (same && (!own_x0 || w.X0.n >= (size_t)slots * N * sizeof(double2))) return RSN_OK;
  const size_t vb = (size_t)slots * N;
  if (own_x0) RSN_CUDA(c, w.X0.ensure(vb * sizeof(double2)));
  if (adjoint) RSN_CUDA(c, w.X1.ensure(vb * sizeof(double2)));
  RSN_CUDA(c, w.r.ensure(vb * el));
  RSN_CUDA(c, w.p0.ensure(vb * el));
  RSN_CUDA(c, w.p1.ensure(vb * el));
  RSN_CUDA(c, w.q.ensure(vb * el));
  RSN_CUDA(c, w.d.ensure(vb * el));
  const size_t si = slots * sizeof(int), sd = slots * sizeof(double);
  RSN_CUDA(c, w.junc.ensure(si));
  RSN_CUDA(c, w.E.ensure(sd));
  RSN_CUDA(c, w.col.ensure(si));
  RSN_CUDA(c, w.voff.ensure(slots * sizeof(long long)));
  RSN_CUDA(c, w.iters.ensure(si));
  RSN_CUDA(c, w.done.ensure(si));
  RSN_CUDA(c, w.outer_done.ensure(si));
  RSN_CUDA(c, w.total_iters.ensure(si));
  RSN_CUDA(c, w.n_outer.ensure(si));
  RSN_CUDA(c, w.status.ensure(si));
  RSN_CUDA(c, w.breakdowns.ensure(si));
  RSN_CUDA(c, w.bnorm2.ensure(sd));
  RSN_CUDA(c, w.tol2.ensure(sd));
  RSN_CUDA(c, w.relres.ensure(sd));
  RSN_CUDA(c, w.out_index.ensure(si));
  RSN_CUDA(c, w.wt.ensure(sd));
  RSN_CUDA(c, w.rho0.ensure((size_t)slots * PA * sizeof(double2)));
  RSN_CUDA(c, w.nrm0.ensure((size_t)slots * PA * sizeof(double)));
  RSN_CUDA(c, w.mu.ensure((size_t)slots * PA * sizeof(double2)));
  RSN_CUDA(c, w.rho.ensure(2 * (size_t)slots * PB * sizeof(double2)));
  RSN_CUDA(c, w.nrm.ensure((size_t)slots * PB * sizeof(double)));
  const size_t npj = std::max(1, c->n_proj);
  RSN_CUDA(c, w.c_r.ensure((size_t)slots * npj * sizeof(double2)));
  RSN_CUDA(c, w.c_p.ensure(2 * (size_t)slots * npj * sizeof(double2)));
  RSN_CUDA(c, w.c_x.ensure((size_t)slots * npj * sizeof(double2)));
  RSN_CUDA(c, w.n_active.ensure(4 * sizeof(int)));
  w.slots = slots;
  w.fp32 = fp32;
  w.adjoint = w.adjoint || adjoint;
  w.N = N;
  w.PA = PA;
  w.PB = PB;
  w.n_proj = c->n_proj;
  w.generation++;
  clear_graphs(c);
  return RSN_OK;
}

static BatchDev batch_view(rsn_ctx* c, double2* x64, const double2* xf) {
  Workspace& w = c->ws;
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.nslots = w.slots;
  b.PA = w.PA;
  b.PB = w.PB;
  b.junc = w.junc.as<int>();
  b.E = w.E.as<double>();
  b.col = w.col.as<int>();
  b.voff = w.voff.as<long long>();
  b.x64 = x64;
  b.xf = xf;
  b.r = w.r.p;
  b.p0 = w.p0.p;
  b.p1 = w.p1.p;
  b.q = w.q.p;
  b.d = w.d.p;
  b.iters = w.iters.as<int>();
  b.done = w.done.as<int>();
  b.outer_done = w.outer_done.as<int>();
  b.total_iters = w.total_iters.as<int>();
  b.n_outer = w.n_outer.as<int>();
  b.status = w.status.as<int>();
  b.breakdowns = w.breakdowns.as<int>();
  b.bnorm2 = w.bnorm2.as<double>();
  b.tol2 = w.tol2.as<double>();
  b.relres = w.relres.as<double>();
  b.rho0_part = w.rho0.as<double2>();
  b.nrm0_part = w.nrm0.as<double>();
  b.rho_part = w.rho.as<double2>();
  b.nrm_part = w.nrm.as<double>();
  b.mu_part = w.mu.as<double2>();
  b.c_r = w.c_r.p;
  b.c_p = w.c_p.p;
  b.c_x = w.c_x.as<double2>();
  b.n_active = w.n_active.as<int>();
  return b;
}

// ---------------------------------------------------------------------------
// one batch: systems [0, nact) of the workspace, slot s with energy E[s] and
// right-hand side col[s] (>= 0: unit vector, -1: adjoint from xf)
// ---------------------------------------------------------------------------
struct BatchResult {
  std::vector<int> total_iters, status, outer_done, n_outer;
  std::vector<double> relres;
  bool timeout = false;
};

static rsn_status run_batch(rsn_ctx* c, const rsn_solver_opts* o, int nact, const double* E, const int* col,
                            double2* x64, const double2* xf, std::chrono::steady_clock::time_point t_start,
                            BatchResult& res) {
  Workspace& w = c->ws;
  const int S = w.slots;
  const bool fp32 = o->precision == RSN_MIXED;
  const long long N = c->N;
  cudaStream_t st = c->st;
  // per-slot inputs
  std::vector<double> hE(S, 0.0), hb(S, 1.0);
  std::vector<int> hcol(S, 0), hj(S, 0), hdone(S, 1), hzero(S, 0);
  std::vector<long long> hvo(S, 0);
  for (int s = 0; s < S; ++s) {
    hvo[s] = (long long)s * N;
    if (s < nact) {
      hE[s] = E[s];
      hcol[s] = col[s];
      hdone[s] = 0;
    }
  }
  RSN_CUDA(c, cudaMemcpyAsync(w.E.p, hE.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.col.p, hcol.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.junc.p, hj.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.voff.p, hvo.data(), S * sizeof(long long), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.done.p, hdone.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.outer_done.p, hdone.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemcpyAsync(w.bnorm2.p, hb.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
  RSN_CUDA(c, cudaMemsetAsync(w.iters.p, 0, S * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.total_iters.p, 0, S * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.n_outer.p, 0, S * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.status.p, 0, S * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.breakdowns.p, 0, S * sizeof(int), st));
  RSN_CUDA(c, cudaMemsetAsync(w.relres.p, 0, S * sizeof(double), st));
  const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
  RSN_CUDA(c, cudaMemsetAsync(x64, 0, (size_t)nact * N * sizeof(double2), st));
  RSN_CUDA(c, cudaMemsetAsync(w.d.p, 0, (size_t)S * N * el, st));

  LaunchCfg cfg;
  rsn_status rs = make_cfg(c, fp32, S, cfg);
  if (rs != RSN_OK) return rs;
  const BatchDev b = batch_view(c, x64, xf);
  const JuncDev* ji = cfg.jt_inner;
  const JuncDev* jr = cfg.jt_resid;
  const int nB = c->jh.nB;
  const bool proj = c->n_proj > 0;
  const dim3 gi(cfg.inner.n, S), gr(cfg.resid.n, S);
  int64_t launches = 0;

  if (xf) {
    RSN_CUDA(c, launch_bnorm_adjoint(S, st, jr, b));
    ++launches;
  }

  auto body = [&](int iters) -> cudaError_t {
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = launch_op(OP_COCG, fp32, c->R, cfg.inner.ppt, gi, cfg.inner.threads, cfg.inner.smem, st, ji, b,
                                nullptr, nullptr, nullptr);
      if (e != cudaSuccess) return e;
      if ((e = launch_cocg_update(fp32, S, nB, st, ji, b)) != cudaSuccess) return e;
      if (proj && (e = launch_project(0, fp32, S, c->n_groups, st, ji, b, nullptr, b.c_r)) != cudaSuccess) return e;
      if ((e = launch_inner_book(S, o->max_iter, st, ji, b)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  const int per_iter = proj ? 4 : 3;
  const int G = std::max(1, o->graph_iters);
  cudaGraphExec_t gexec = nullptr;
  if (o->use_graph) {
    GraphKey key{fp32 ? 1 : 0, S, G, w.generation, proj ? 1 : 0};
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
      gexec = it->second;
    } else {
      cudaGraph_t g = nullptr;
      RSN_CUDA(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = body(G);
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

  bool timeout = false;
  for (int outer = 0; outer <= o->max_outer + 1; ++outer) {
    if (proj) {
      RSN_CUDA(c, launch_project(1, fp32, S, c->n_groups, st, jr, b, nullptr, b.c_x));
      ++launches;
    }
    RSN_CUDA(c, launch_op(OP_RESID, fp32, c->R, cfg.resid.ppt, gr, cfg.resid.threads, cfg.resid.smem, st, jr, b,
                          nullptr, nullptr, nullptr));
    RSN_CUDA(c, launch_x_update(fp32, S, nB, st, jr, b));
    RSN_CUDA(c, launch_outer_book(S, o->tol, o->tol_inner, o->max_outer, st, jr, b));
    launches += 3;
    RSN_CUDA(c, cudaMemcpyAsync(c->n_active_host, b.n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    RSN_CUDA(c, cudaStreamSynchronize(st));
    if (c->n_active_host[1] == 0) break;
    c->st_sweeps++;
    if (proj) {
      RSN_CUDA(c, launch_project(0, fp32, S, c->n_groups, st, ji, b, nullptr, b.c_r));
      ++launches;
    }
    // inner COCG: replay the captured iteration body until no system is active
    for (int rep = 0;; ++rep) {
      if (gexec) {
        RSN_CUDA(c, cudaGraphLaunch(gexec, st));
      } else {
        RSN_CUDA(c, body(G));
      }
      launches += (int64_t)G * per_iter;
      RSN_CUDA(c, cudaMemcpyAsync(c->n_active_host, b.n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      RSN_CUDA(c, cudaStreamSynchronize(st));
      if (c->n_active_host[0] == 0) break;
      if (o->deadline_ms > 0) {
        const double el_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (el_ms > o->deadline_ms) {
          timeout = true;
          break;
        }
      }
      if ((long long)rep * G > (long long)o->max_iter + G) break;  // safety: max_iter bounds every slot
    }
    if (timeout) break;
  }
  c->st_launches += launches;
  res.total_iters.resize(S);
  res.status.resize(S);
  res.outer_done.resize(S);
  res.n_outer.resize(S);
  res.relres.resize(S);
  RSN_CUDA(c, cudaMemcpyAsync(res.total_iters.data(), w.total_iters.p, S * sizeof(int), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(res.status.data(), w.status.p, S * sizeof(int), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(res.outer_done.data(), w.outer_done.p, S * sizeof(int), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(res.n_outer.data(), w.n_outer.p, S * sizeof(int), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaMemcpyAsync(res.relres.data(), w.relres.p, S * sizeof(double), cudaMemcpyDeviceToHost, st));
  RSN_CUDA(c, cudaStreamSynchronize(st));
  res.timeout = timeout;
  return RSN_OK;
}

// classify a finished batch into an overall status; fills iters/relres
static rsn_status batch_status(const BatchResult& r, int nact, double tol, int32_t* iters, double* relres) {
  rsn_status worst = RSN_OK;
  for (int s = 0; s < nact; ++s) {
    const bool ok = r.outer_done[s] && r.status[s] == 0 && r.relres[s] <= tol;
    if (iters) iters[s] = ok ? r.total_iters[s] : -std::max(1, r.total_iters[s]);
    if (relres) relres[s] = r.relres[s];
    if (!ok) {
      rsn_status e = r.timeout ? RSN_ETIMEOUT : (r.status[s] == 2 ? RSN_EBREAKDOWN : RSN_ENOCONV);
      if (worst == RSN_OK) worst = e;
    }
  }
  return worst;
}

static rsn_status check_solve_args(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                   const rsn_solver_opts* o) {
  if (n_e < 0 || n_cols < 0) RSN_FAIL(c, RSN_EINVAL, "negative sizes");
  if ((n_e > 0 && !E) || (n_cols > 0 && !cols) || !o) RSN_FAIL(c, RSN_EINVAL, "NULL argument");
  if (o->precision != RSN_FP64 && o->precision != RSN_MIXED) RSN_FAIL(c, RSN_EINVAL, "bad precision");
  if (!(o->tol > 0) || !(o->tol_inner > 0) || o->max_iter < 1 || o->max_outer < 0)
    RSN_FAIL(c, RSN_EINVAL, "bad solver options");
  for (int e = 0; e < n_e; ++e)
    if (!std::isfinite(E[e])) RSN_FAIL(c, RSN_EINVAL, "E[%d] is not finite", e);
  for (int k = 0; k < n_cols; ++k)
    if (cols[k] < 0 || cols[k] >= c->N) RSN_FAIL(c, RSN_EINVAL, "cols[%d] = %d out of range", k, cols[k]);
  return RSN_OK;
}

extern "C" {

rsn_status rsn_apply(rsn_ctx* c, int precision, int n_rhs, const double* E, const void* x_dev, void* y_dev) {
  if (!c) return RSN_EINVAL;
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if (n_rhs < 0 || (n_rhs > 0 && (!E || !x_dev || !y_dev))) RSN_FAIL(c, RSN_EINVAL, "bad arguments");
  if (precision != RSN_FP64 && precision != RSN_MIXED) RSN_FAIL(c, RSN_EINVAL, "bad precision");
  if (n_rhs == 0) return RSN_OK;
  if ((rs = enter(c)) != RSN_OK) return rs;
  const bool fp32 = precision == RSN_MIXED;
  if ((rs = ensure_ws(c, fp32, false, n_rhs, false)) != RSN_OK) return rs;
  Workspace& w = c->ws;
  std::vector<double> hE(E, E + n_rhs);
  hE.resize(w.slots, 0.0);
  std::vector<int> hj(w.slots, 0);
  std::vector<long long> hvo(w.slots);
  for (int s = 0; s < w.slots; ++s) hvo[s] = (long long)s * c->N;
  RSN_CUDA(c, cudaMemcpyAsync(w.E.p, hE.data(), w.slots * sizeof(double), cudaMemcpyHostToDevice, c->st));
  RSN_CUDA(c, cudaMemcpyAsync(w.junc.p, hj.data(), w.slots * sizeof(int), cudaMemcpyHostToDevice, c->st));
  RSN_CUDA(c, cudaMemcpyAsync(w.voff.p, hvo.data(), w.slots * sizeof(long long), cudaMemcpyHostToDevice, c->st));
  LaunchCfg cfg;
  if ((rs = make_cfg(c, fp32, w.slots, cfg)) != RSN_OK) return rs;
  Tiling t = choose_tiling(c, !fp32, OP_APPLY, w.slots);
  BatchDev b = batch_view(c, nullptr, nullptr);
  b.nslots = n_rhs;
  if (c->n_proj > 0) RSN_CUDA(c, launch_project(2, fp32, n_rhs, c->n_groups, c->st, cfg.jt_inner, b, x_dev, b.c_r));
  RSN_CUDA(c, launch_op(OP_APPLY, fp32, c->R, t.ppt, dim3(cfg.inner.n, n_rhs), t.threads, t.smem, c->st,
                        cfg.jt_inner, b, x_dev, y_dev, b.c_r));
  return leave(c);
}

rsn_status rsn_solve_columns(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                             const rsn_solver_opts* o, void* x_dev, int32_t* iters, double* relres) {
  if (!c) return RSN_EINVAL;
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((rs = check_solve_args(c, n_e, E, n_cols, cols, o)) != RSN_OK) return rs;
  const long long total = (long long)n_e * n_cols;
  if (total == 0) return RSN_OK;
  if (!x_dev) RSN_FAIL(c, RSN_EINVAL, "x_dev is NULL");
  if ((rs = enter(c)) != RSN_OK) return rs;
  const bool fp32 = o->precision == RSN_MIXED;
  const int S = choose_slots(c, o, false, total);
  if ((rs = ensure_ws(c, fp32, false, S, false)) != RSN_OK) return rs;
  c->st_iters = c->st_sweeps = c->st_launches = 0;
  const auto t_start = std::chrono::steady_clock::now();
  RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
  rsn_status worst = RSN_OK;
  std::vector<double> bE(S);
  std::vector<int> bc(S);
  for (long long s0 = 0; s0 < total; s0 += S) {
    const int nact = (int)std::min<long long>(S, total - s0);
    for (int s = 0; s < nact; ++s) {
      bE[s] = E[(s0 + s) / n_cols];
      bc[s] = cols[(s0 + s) % n_cols];
    }
    double2* x64 = reinterpret_cast<double2*>(x_dev) + s0 * c->N;
    BatchResult br;
    if ((rs = run_batch(c, o, nact, bE.data(), bc.data(), x64, nullptr, t_start, br)) != RSN_OK) return rs;
    for (int s = 0; s < nact; ++s) c->st_iters += br.total_iters[s];
    rsn_status bs = batch_status(br, nact, o->tol, iters ? iters + s0 : nullptr, relres ? relres + s0 : nullptr);
    if (worst == RSN_OK) worst = bs;
  }
  RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
  RSN_CUDA(c, cudaEventSynchronize(c->t1));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->t0, c->t1);
  c->st_ms = ms;
  if ((rs = leave(c)) != RSN_OK) return rs;
  if (worst != RSN_OK) RSN_FAIL(c, worst, "some columns did not reach tol (status %d)", (int)worst);
  return RSN_OK;
}

// Shared driver of rsn_transmission and rsn_transmission_vjp.
static rsn_status transmission_impl(rsn_ctx* c, int n_e, const double* E, int n_cols, const int32_t* cols,
                                    const rsn_solver_opts* o, const double* T_bar, double* dV, int dV_dev,
                                    double* T) {
  rsn_status rs = commit_setup(c);
  if (rs != RSN_OK) return rs;
  if ((rs = check_solve_args(c, n_e, E, n_cols, cols, o)) != RSN_OK) return rs;
  const bool adjoint = dV != nullptr;
  if (adjoint && n_e > 0 && !T_bar) RSN_FAIL(c, RSN_EINVAL, "T_bar is NULL");
  if ((rs = enter(c)) != RSN_OK) return rs;
  const long long total = (long long)n_e * n_cols;
  const bool fp32 = o->precision == RSN_MIXED;
  c->st_iters = c->st_sweeps = c->st_launches = 0;
  DevBuf t_all, gr_cols, Td, g, oi;
  RSN_CUDA(c, t_all.ensure(std::max<long long>(1, total) * sizeof(double)));
  RSN_CUDA(c, gr_cols.ensure(std::max(1, n_cols) * sizeof(double)));
  RSN_CUDA(c, Td.ensure(std::max(1, n_e) * sizeof(double)));
  if (adjoint) {
    RSN_CUDA(c, g.ensure(c->N * sizeof(double)));
    RSN_CUDA(c, cudaMemsetAsync(g.p, 0, c->N * sizeof(double), c->st));
  }
  std::vector<double> hgr(std::max(1, n_cols));
  for (int k = 0; k < n_cols; ++k) hgr[k] = c->gr[cols[k]];
  RSN_CUDA(c, cudaMemcpyAsync(gr_cols.p, hgr.data(), hgr.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  const auto t_start = std::chrono::steady_clock::now();
  RSN_CUDA(c, cudaEventRecord(c->t0, c->st));
  rsn_status worst = RSN_OK;
  if (total > 0) {
    const int S = choose_slots(c, o, adjoint, total);
    if ((rs = ensure_ws(c, fp32, adjoint, S, true)) != RSN_OK) return rs;
    Workspace& w = c->ws;
    std::vector<double> bE(S), hw(S);
    std::vector<int> bc(S), hoi(S), bcadj(S, -1);
    for (long long s0 = 0; s0 < total; s0 += S) {
      const int nact = (int)std::min<long long>(S, total - s0);
      for (int s = 0; s < S; ++s) {
        if (s < nact) {
          bE[s] = E[(s0 + s) / n_cols];
          bc[s] = cols[(s0 + s) % n_cols];
          hoi[s] = (int)(s0 + s);
          hw[s] = adjoint ? 8.0 * c->gr[bc[s]] * T_bar[(s0 + s) / n_cols] : 0.0;
        } else {
          hoi[s] = -1;
          hw[s] = 0.0;
        }
      }
      BatchResult br;
      double2* X0 = w.X0.as<double2>();
      if ((rs = run_batch(c, o, nact, bE.data(), bc.data(), X0, nullptr, t_start, br)) != RSN_OK) return rs;
      for (int s = 0; s < nact; ++s) c->st_iters += br.total_iters[s];
      rsn_status bs = batch_status(br, nact, o->tol, nullptr, nullptr);
      if (worst == RSN_OK) worst = bs;
      RSN_CUDA(c, cudaMemcpyAsync(w.out_index.p, hoi.data(), S * sizeof(int), cudaMemcpyHostToDevice, c->st));
      BatchDev bv = batch_view(c, X0, nullptr);
      LaunchCfg cfg;
      if ((rs = make_cfg(c, fp32, S, cfg)) != RSN_OK) return rs;
      RSN_CUDA(c, launch_t_partial(S, c->st, cfg.jt_inner, bv, w.out_index.as<int>(), t_all.as<double>()));
      c->st_launches += 1;
      if (adjoint) {
        BatchResult ba;
        double2* X1 = w.X1.as<double2>();
        if ((rs = run_batch(c, o, nact, bE.data(), bcadj.data(), X1, X0, t_start, ba)) != RSN_OK) return rs;
        for (int s = 0; s < nact; ++s) c->st_iters += ba.total_iters[s];
        bs = batch_status(ba, nact, o->tol, nullptr, nullptr);
        if (worst == RSN_OK) worst = bs;
        RSN_CUDA(c, cudaMemcpyAsync(w.wt.p, hw.data(), S * sizeof(double), cudaMemcpyHostToDevice, c->st));
        BatchDev ba_v = batch_view(c, X1, X0);
        RSN_CUDA(c, launch_grad_accum(S, c->N, c->st, ba_v, w.wt.as<double>(), g.as<double>()));
        c->st_launches += 1;
      }
    }
  }
  RSN_CUDA(c, launch_t_final(n_e, n_cols, c->st, t_all.as<double>(), gr_cols.as<double>(), Td.as<double>()));
  c->st_launches += 1;
  RSN_CUDA(c, cudaEventRecord(c->t1, c->st));
  if (T && n_e > 0) RSN_CUDA(c, cudaMemcpyAsync(T, Td.p, n_e * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if (adjoint) {
    RSN_CUDA(c, cudaMemcpyAsync(dV, g.p, c->N * sizeof(double),
                                dV_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  }
  RSN_CUDA(c, cudaStreamSynchronize(c->st));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->t0, c->t1);
  c->st_ms = ms;
  if ((rs = leave(c)) != RSN_OK) return rs;
  if (worst != RSN_OK) RSN_FAIL(c, worst, "some columns did not reach tol (status %d)", (int)worst);
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

// Tiling override used by the autotuner and the tests: TY, Lz, ppt (0 = auto).
rsn_status rsn_set_tiling(rsn_ctx* c, int TY, int Lz, int ppt) {
  if (!c) return RSN_EINVAL;
  if (TY < 0 || Lz < 0 || ppt < 0 || ppt > 4) RSN_FAIL(c, RSN_EINVAL, "bad tiling override");
  c->tile_override[0] = TY;
  c->tile_override[1] = Lz;
  c->tile_override[2] = ppt;
  clear_graphs(c);
  c->ws.generation++;
  c->ws.slots = 0;  // partial strides may change
  return RSN_OK;
}

}  // extern "C"
