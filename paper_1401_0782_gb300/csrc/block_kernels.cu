// Block COCG kernels: the B right-hand sides e_j of one energy share one block
// Krylov space of A(E) = E - H + i Gamma (Eqs. G, Hop; A = A^T by Eq.
// complex-sym, so the unconjugated bilinear form u^T v replaces the inner
// product of block CG).  The residual block is kept orthonormal:
//
//   R_k = Q_k xi_k,  Q_k = W_k tau_k^{-1}  (Cholesky QR: W_k^H W_k = tau_k^H tau_k)
//   P_k = Q_k + P_{k-1} beta_{k-1}                    (P_0 = Q_0)
//   alpha_k = (P_k^T A P_k)^{-1} (Q_k^T Q_k)
//   D += P_k alpha_k xi_k
//   W_{k+1} = Q_k - A P_k alpha_k,   tau_{k+1} from W_{k+1},   xi_{k+1} = tau_{k+1} xi_k
//   beta_k = (Q_k^T Q_k)^{-1} tau_{k+1}^T (Q_{k+1}^T Q_{k+1})
//
// and ||r_j|| = ||xi[:, j]|| because Q is orthonormal.  One inner iteration:
//   comb_p   P = W tau^{-1} + P beta                     (vectors, FP32)
//   project + operator (the apply kernels)   AP = A P
//   gram 0   partial sums of P^T AP                      (b x b, FP32 products)
//   small 1  alpha, alpha xi                             (b x b, FP64, one warp per block)
//   comb_w   W = W tau^{-1} - AP alpha,  D += P alpha xi (vectors, FP32)
//   gram 1   partial sums of W^H W and W^T W
//   small 2  tau, tau^{-1}, xi, Q^T Q, beta; convergence
// A restart (start of an inner solve on the normalised FP64 residual block Rh)
// takes its QR in FP64: gram64 (Rh^H Rh, Rh^T Rh), small 0 (tau_0, xi_0 = tau_0,
// Q_0^T Q_0), q0 (W = Q_0 = Rh tau_0^{-1}, rounded once).
// Every kernel skips blocks whose flag is set (converged, breakdown, cap).
#include <cfloat>

#include "cplx.cuh"
#include "rsn_internal.h"

namespace rsn {

namespace {

__device__ __forceinline__ float2 cfma_f(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  return acc;
}
// acc + conj(a) b
__device__ __forceinline__ float2 cjfma_f(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
  return acc;
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 to32(double2 a) { return make_float2((float)a.x, (float)a.y); }

// Sums of FP32 products to about FP64 accuracy in FP32 arithmetic: each
// product a b is split exactly into p = fl(a b) and its rounding error
// e = fma(a, b, -p) (error-free transformation); the p are summed with Kahan's
// compensation, the e plainly (they are ~1e-7 of the p).  The explicit _rn
// intrinsics keep the compiler from contracting p into a later addition.
struct KSum {
  float s, c, e;
};
__device__ __forceinline__ void ks_add(KSum& k, float a, float b) {
  const float p = __fmul_rn(a, b);
  k.e = __fadd_rn(k.e, __fmaf_rn(a, b, -p));
  const float y = __fsub_rn(p, k.c);
  const float t = __fadd_rn(k.s, y);
  k.c = __fsub_rn(__fsub_rn(t, k.s), y);
  k.s = t;
}
__device__ __forceinline__ double ks_val(const KSum& k) { return (double)k.s - (double)k.c + (double)k.e; }

}  // namespace

// ---------------------------------------------------------------------------
// P = W tau^{-1} + P beta   (P = W tau^{-1} in the first iteration)
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(kBlkThreads) blk_comb_p_kernel(const BlkDev* __restrict__ dp) {
  const BlkDev& d = *dp;
  const int k = d.blist[blockIdx.y];
  if (d.flag[k] != 0) return;
  __shared__ float2 sT[B * B], sB[B * B];
  const bool first = d.its[k] == 0;
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    sT[e] = d.tinv[(size_t)k * B * B + e];
    sB[e] = first ? make_float2(0.f, 0.f) : d.beta[(size_t)k * B * B + e];
  }
  __syncthreads();
  const long long N = d.N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const size_t base = (size_t)k * B * N + i;
  float2 w[B], p[B];
#pragma unroll
  for (int a = 0; a < B; ++a) w[a] = d.W[base + (size_t)a * N];
  if (!first) {
#pragma unroll
    for (int a = 0; a < B; ++a) p[a] = d.P[base + (size_t)a * N];
  } else {
#pragma unroll
    for (int a = 0; a < B; ++a) p[a] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int c = 0; c < B; ++c) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a <= c; ++a) acc = cfma_f(w[a], sT[a * B + c], acc);  // tau^{-1} upper triangular
    if (!first) {
#pragma unroll
      for (int a = 0; a < B; ++a) acc = cfma_f(p[a], sB[a * B + c], acc);
    }
    d.P[base + (size_t)c * N] = acc;
  }
}

// ---------------------------------------------------------------------------
// W = W tau^{-1} - AP alpha,   D += P (alpha xi)
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(kBlkThreads) blk_comb_w_kernel(const BlkDev* __restrict__ dp) {
  const BlkDev& d = *dp;
  const int k = d.blist[blockIdx.y];
  if (d.flag[k] != 0) return;
  __shared__ float2 sT[B * B], sA[B * B], sX[B * B];
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    sT[e] = d.tinv[(size_t)k * B * B + e];
    const float2 a = d.alpha[(size_t)k * B * B + e];
    sA[e] = make_float2(-a.x, -a.y);
    sX[e] = d.axi[(size_t)k * B * B + e];
  }
  __syncthreads();
  const long long N = d.N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const size_t base = (size_t)k * B * N + i;
  {
    float2 w[B], q[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      w[a] = d.W[base + (size_t)a * N];
      q[a] = d.AP[base + (size_t)a * N];
    }
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a <= c; ++a) acc = cfma_f(w[a], sT[a * B + c], acc);
#pragma unroll
      for (int a = 0; a < B; ++a) acc = cfma_f(q[a], sA[a * B + c], acc);
      d.W[base + (size_t)c * N] = acc;  // every member of this point was read above
    }
  }
  {
    float2 p[B];
#pragma unroll
    for (int a = 0; a < B; ++a) p[a] = d.P[base + (size_t)a * N];
#pragma unroll
    for (int c = 0; c < B; ++c) {
      float2 acc = d.D[base + (size_t)c * N];
#pragma unroll
      for (int a = 0; a < B; ++a) acc = cfma_f(p[a], sX[a * B + c], acc);
      d.D[base + (size_t)c * N] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Gram partial sums over one chunk of points of each listed block.
// MODE 0: U = P, V = AP, out[0] = U^T V.   MODE 1: U = V = W, out[0] = W^H W,
// out[1] = W^T W.  Tiles of kBlkTile points of every member are staged in
// shared memory (row pitch kBlkTile + 1 keeps the members' rows on distinct
// banks); each thread owns a 2 x 2 tile of (a, c) pairs and a slice of the
// tile's points.  The sums reach about FP64 accuracy in FP32 arithmetic
// (error-free products, compensated sums; the point slices and chunks in
// FP64): the block recurrence's b x b systems come from Gram matrices of
// nearly dependent directions once its residual columns share the slowest
// modes of A(E), and FP32 sums of them stall its restarts.
// ---------------------------------------------------------------------------
template <int B, int MODE>
__global__ void __launch_bounds__(kBlkThreads) blk_gram_kernel(const BlkDev* __restrict__ dp) {
  constexpr int H = B / 2;
  constexpr int NT = H * H;                // pair tiles
  constexpr int PG = kBlkThreads / NT;     // point slices
  constexpr int TP = kBlkTile;
  constexpr int LD = TP + 1;
  constexpr int NO = MODE == 0 ? 1 : 2;    // outputs
  static_assert(PG >= 1 && TP % PG == 0, "tile split");
  const BlkDev& d = *dp;
  const int k = d.blist[blockIdx.y];
  if (d.flag[k] != 0) return;
  __shared__ float2 sU[B * LD];
  __shared__ float2 sV[(MODE == 0 ? B : 1) * LD];
  __shared__ double2 red[PG * NT * 4 * NO];
  const long long N = d.N;
  const int chunk = blockIdx.x;
  const long long x0 = (long long)chunk * d.chunk_pts;
  const long long x1 = min(N, x0 + d.chunk_pts);
  const size_t base = (size_t)k * B * N;
  const float2* U = MODE == 0 ? d.P : d.W;
  const float2* V = MODE == 0 ? d.AP : d.W;
  const int tid = threadIdx.x;
  const int t = tid % NT, g = tid / NT;
  const int a0 = 2 * (t / H), c0 = 2 * (t % H);
  // [output][pair][re, im]
  KSum ks[NO][4][2];
#pragma unroll
  for (int o = 0; o < NO; ++o)
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int r = 0; r < 2; ++r) ks[o][m][r] = KSum{0.f, 0.f, 0.f};
  for (long long ts = x0; ts < x1; ts += TP) {
    for (int e = tid; e < B * TP; e += kBlkThreads) {
      const int a = e / TP, ii = e % TP;
      const long long i = ts + ii;
      const bool in = i < x1;
      sU[a * LD + ii] = in ? U[base + (size_t)a * N + i] : make_float2(0.f, 0.f);
      if constexpr (MODE == 0) sV[a * LD + ii] = in ? V[base + (size_t)a * N + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* sv = MODE == 0 ? sV : sU;
#pragma unroll 2
    for (int ii = g; ii < TP; ii += PG) {
      const float2 uu[2] = {sU[a0 * LD + ii], sU[(a0 + 1) * LD + ii]};
      const float2 vv[2] = {sv[c0 * LD + ii], sv[(c0 + 1) * LD + ii]};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 u = uu[m >> 1], v = vv[m & 1];
        if constexpr (MODE == 0) {
          // u v
          ks_add(ks[0][m][0], u.x, v.x);
          ks_add(ks[0][m][0], -u.y, v.y);
          ks_add(ks[0][m][1], u.x, v.y);
          ks_add(ks[0][m][1], u.y, v.x);
        } else {
          // conj(u) v and u v
          ks_add(ks[0][m][0], u.x, v.x);
          ks_add(ks[0][m][0], u.y, v.y);
          ks_add(ks[0][m][1], u.x, v.y);
          ks_add(ks[0][m][1], -u.y, v.x);
          ks_add(ks[1][m][0], u.x, v.x);
          ks_add(ks[1][m][0], -u.y, v.y);
          ks_add(ks[1][m][1], u.x, v.y);
          ks_add(ks[1][m][1], u.y, v.x);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 0; o < NO; ++o)
#pragma unroll
    for (int m = 0; m < 4; ++m)
      red[((o * PG + g) * NT + t) * 4 + m] = make_double2(ks_val(ks[o][m][0]), ks_val(ks[o][m][1]));
  __syncthreads();
  // slices summed in a fixed order; entry (a, c) of output o
  double2* out = d.part + ((size_t)k * d.nchunk + chunk) * 2 * B * B;
  for (int e = tid; e < NO * B * B; e += kBlkThreads) {
    const int o = e / (B * B), ac = e % (B * B);
    const int a = ac / B, c = ac % B;
    const int tt = (a / 2) * H + (c / 2), m = (a & 1) * 2 + (c & 1);
    double2 v = make_double2(0.0, 0.0);
    for (int gg = 0; gg < PG; ++gg) {
      const double2 r = red[((o * PG + gg) * NT + tt) * 4 + m];
      v.x += r.x;
      v.y += r.y;
    }
    out[(size_t)o * B * B + ac] = v;
  }
}

// ---------------------------------------------------------------------------
// Restart of an inner solve: partial sums of Rh^H Rh and Rh^T Rh of the
// normalised FP64 residual block Rh = R / ||R|| (in R), products and sums in
// FP64.  The residual columns of a restart share the slowest modes of A(E) and
// are close to dependent; an FP32 Gram would lose the orthogonality of Q_0 to
// rounding (~1e-7 kappa^2), the FP64 one keeps it.  Same layout as the FP32
// Gram: a 2 x 2 tile of (a, c) pairs per thread over a slice of the points.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(kBlkThreads) blk_gram64_kernel(const BlkDev* __restrict__ dp) {
  constexpr int H = B / 2;
  constexpr int NT = H * H;
  constexpr int PG = kBlkThreads / NT;
  const BlkDev& d = *dp;
  const int k = d.blist[blockIdx.y];
  if (d.flag[k] != 0) return;
  __shared__ double2 red[PG * NT * 4 * 2];
  const long long N = d.N;
  const int chunk = blockIdx.x;
  const long long x0 = (long long)chunk * d.chunk_pts;
  const long long x1 = min(N, x0 + d.chunk_pts);
  const double2* R = d.R + (size_t)k * B * N;
  const int tid = threadIdx.x;
  const int t = tid % NT, g = tid / NT;
  const int a0 = 2 * (t / H), c0 = 2 * (t % H);
  double2 sh[4], st[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) sh[m] = st[m] = make_double2(0.0, 0.0);
  for (long long i = x0 + g; i < x1; i += PG) {
    const double2 u0 = R[(size_t)a0 * N + i], u1 = R[(size_t)(a0 + 1) * N + i];
    const double2 v0 = R[(size_t)c0 * N + i], v1 = R[(size_t)(c0 + 1) * N + i];
    const double2 uu[2] = {u0, u1}, vv[2] = {v0, v1};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double2 u = uu[m >> 1], v = vv[m & 1];
      sh[m].x += u.x * v.x + u.y * v.y;  // conj(u) v
      sh[m].y += u.x * v.y - u.y * v.x;
      st[m].x += u.x * v.x - u.y * v.y;  // u v
      st[m].y += u.x * v.y + u.y * v.x;
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    red[((0 * PG + g) * NT + t) * 4 + m] = sh[m];
    red[((1 * PG + g) * NT + t) * 4 + m] = st[m];
  }
  __syncthreads();
  double2* out = d.part + ((size_t)k * d.nchunk + chunk) * 2 * B * B;
  for (int e = tid; e < 2 * B * B; e += kBlkThreads) {
    const int o = e / (B * B), ac = e % (B * B);
    const int a = ac / B, c = ac % B;
    const int tt = (a / 2) * H + (c / 2), m = (a & 1) * 2 + (c & 1);
    double2 v = make_double2(0.0, 0.0);
    for (int gg = 0; gg < PG; ++gg) {
      const double2 r = red[((o * PG + gg) * NT + tt) * 4 + m];
      v.x += r.x;
      v.y += r.y;
    }
    out[(size_t)o * B * B + ac] = v;
  }
}

// Q_0 = Rh tau_0^{-1} in FP64 (tau_0^{-1} from the restart's Cholesky, upper
// triangular), rounded to FP32 into W; D = 0.
template <int B>
__global__ void __launch_bounds__(kBlkThreads) blk_q0_kernel(const BlkDev* __restrict__ dp) {
  const BlkDev& d = *dp;
  const int k = d.blist[blockIdx.y];
  if (d.flag[k] != 0) return;
  __shared__ double2 sT[B * B];
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) sT[e] = d.tinv64[(size_t)k * B * B + e];
  __syncthreads();
  const long long N = d.N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const size_t base = (size_t)k * B * N + i;
  double2 r[B];
#pragma unroll
  for (int a = 0; a < B; ++a) r[a] = d.R[base + (size_t)a * N];
#pragma unroll
  for (int c = 0; c < B; ++c) {
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int a = 0; a <= c; ++a) {
      const double2 t = sT[a * B + c];
      acc.x += r[a].x * t.x - r[a].y * t.y;
      acc.y += r[a].x * t.y + r[a].y * t.x;
    }
    d.W[base + (size_t)c * N] = make_float2((float)acc.x, (float)acc.y);
    d.D[base + (size_t)c * N] = make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
// b x b algebra, one warp per listed block, FP64.
// ---------------------------------------------------------------------------
namespace {

// Sum the Gram partials of output o over the chunks into M (row-major B x B,
// leading dimension ld).
template <int B>
__device__ void sum_parts(const BlkDev& d, int k, int o, double2* M, int ld) {
  const int lane = threadIdx.x;
  for (int e = lane; e < B * B; e += 32) {
    double2 v = make_double2(0.0, 0.0);
    for (int ch = 0; ch < d.nchunk; ++ch) {
      const double2 r = d.part[(((size_t)k * d.nchunk + ch) * 2 + o) * B * B + e];
      v.x += r.x;
      v.y += r.y;
    }
    M[(e / B) * ld + (e % B)] = v;
  }
  __syncwarp();
}

// Solve M X = Y for the B x B block X, with M and Y held side by side in
// aug (B rows, 2B columns, leading dimension 2B): Gaussian elimination with
// partial pivoting, lane j owning augmented column j.  The solution goes to
// sol (row-major B x B).  Returns false on a zero or non-finite pivot.
template <int B>
__device__ bool warp_solve(double2* aug, double2* fac, int* s_piv, double2* sol) {
  constexpr int L = 2 * B;
  const int lane = threadIdx.x;
  bool ok = true;
  for (int kk = 0; kk < B; ++kk) {
    if (lane == 0) {
      int piv = kk;
      double best = cabs2(aug[kk * L + kk]);
      for (int r = kk + 1; r < B; ++r) {
        const double v = cabs2(aug[r * L + kk]);
        if (v > best) best = v, piv = r;
      }
      *s_piv = (best > 0.0 && best <= DBL_MAX) ? piv : -1;
    }
    __syncwarp();
    const int piv = *s_piv;
    if (piv < 0) {
      ok = false;
      break;
    }
    if (piv != kk && lane < L) {
      const double2 tmp = aug[kk * L + lane];
      aug[kk * L + lane] = aug[piv * L + lane];
      aug[piv * L + lane] = tmp;
    }
    __syncwarp();
    if (lane > kk && lane < B) fac[lane] = cdiv(aug[lane * L + kk], aug[kk * L + kk]);
    __syncwarp();
    if (lane > kk && lane < L) {
      const double2 top = aug[kk * L + lane];
      for (int r = kk + 1; r < B; ++r) {
        const double2 f = fac[r];
        double2 v = aug[r * L + lane];
        v.x -= f.x * top.x - f.y * top.y;
        v.y -= f.x * top.y + f.y * top.x;
        aug[r * L + lane] = v;
      }
    }
    __syncwarp();
  }
  if (!ok) return false;
  if (lane >= B && lane < L) {
    const int j = lane - B;
    for (int r = B - 1; r >= 0; --r) {
      double2 v = aug[r * L + lane];
      for (int m = r + 1; m < B; ++m) {
        const double2 a = aug[r * L + m], x = sol[m * B + j];
        v.x -= a.x * x.x - a.y * x.y;
        v.y -= a.x * x.y + a.y * x.x;
      }
      sol[r * B + j] = cdiv(v, aug[r * L + r]);
    }
  }
  __syncwarp();
  return true;
}

// Cholesky factor of the Hermitian positive definite A (row-major B x B):
// A = Lc Lc^H, Lc lower triangular with a real positive diagonal; lanes own
// rows.  Fails when a pivot is not positive or falls below 1e-12 of its
// diagonal entry (numerically dependent columns).
template <int B>
__device__ bool warp_cholesky(const double2* A, double2* Lc, int* s_ok) {
  const int lane = threadIdx.x;
  for (int e = lane; e < B * B; e += 32) Lc[e] = make_double2(0.0, 0.0);
  if (lane == 0) *s_ok = 1;
  __syncwarp();
  for (int kk = 0; kk < B; ++kk) {
    if (lane == 0) {
      double dd = A[kk * B + kk].x;
      for (int m = 0; m < kk; ++m) dd -= cabs2(Lc[kk * B + m]);
      const double ref = A[kk * B + kk].x;
      if (!(dd > 1e-12 * ref) || !(dd <= DBL_MAX)) {
        *s_ok = 0;
        dd = 1.0;
      }
      Lc[kk * B + kk] = make_double2(sqrt(dd), 0.0);
    }
    __syncwarp();
    if (lane > kk && lane < B) {
      double2 v = A[lane * B + kk];
      for (int m = 0; m < kk; ++m) {
        const double2 a = Lc[lane * B + m], b = Lc[kk * B + m];  // a conj(b)
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
      }
      const double dk = Lc[kk * B + kk].x;
      Lc[lane * B + kk] = make_double2(v.x / dk, v.y / dk);
    }
    __syncwarp();
  }
  return *s_ok != 0;
}

// Li = Lc^{-1} (lower triangular), lane j owning column j.
template <int B>
__device__ void warp_lower_inverse(const double2* Lc, double2* Li) {
  const int j = threadIdx.x;
  if (j < B) {
    for (int r = 0; r < B; ++r) {
      double2 v = make_double2(r == j ? 1.0 : 0.0, 0.0);
      if (r > j) {
        v = make_double2(0.0, 0.0);
        for (int m = j; m < r; ++m) {
          const double2 a = Lc[r * B + m], x = Li[m * B + j];
          v.x -= a.x * x.x - a.y * x.y;
          v.y -= a.x * x.y + a.y * x.x;
        }
      }
      const double dr = Lc[r * B + r].x;
      Li[r * B + j] = r < j ? make_double2(0.0, 0.0) : make_double2(v.x / dr, v.y / dr);
    }
  }
  __syncwarp();
}

// C = A Bm for row-major B x B matrices, lane j owning column j of C.
template <int B>
__device__ void warp_matmul(const double2* A, const double2* Bm, double2* C) {
  const int j = threadIdx.x;
  if (j < B) {
    for (int r = 0; r < B; ++r) {
      double2 v = make_double2(0.0, 0.0);
      for (int m = 0; m < B; ++m) {
        const double2 a = A[r * B + m];
        const double2 b = Bm[m * B + j];
        v.x += a.x * b.x - a.y * b.y;
        v.y += a.x * b.y + a.y * b.x;
      }
      C[r * B + j] = v;
    }
  }
  __syncwarp();
}

}  // namespace

// PHASE 0: start of an inner solve (W holds the normalised residual block):
//          tau_0, tau_0^{-1}, xi_0 = tau_0, ||xi_0[:, j]||, Q_0^T Q_0.
// PHASE 1: alpha = (P^T AP)^{-1} Q^T Q and alpha xi.
// PHASE 2: tau, tau^{-1} of the new W; xi <- tau xi; Q^T Q of the new Q;
//          beta; iteration count and convergence of every column.
template <int B, int PHASE>
__global__ void __launch_bounds__(32) blk_small_kernel(const BlkDev* __restrict__ dp) {
  const BlkDev& d = *dp;
  const int k = d.blist[blockIdx.x];
  const int lane = threadIdx.x;
  if (PHASE != 0 && d.flag[k] != 0) return;
  __shared__ double2 aug[B * 2 * B];
  __shared__ double2 M0[B * B], M1[B * B], M2[B * B], M3[B * B];
  __shared__ double2 fac[B];
  __shared__ int s_i;
  const size_t ko = (size_t)k * B * B;
  if (PHASE == 1) {
    sum_parts<B>(d, k, 0, aug, 2 * B);  // P^T A P
    for (int e = lane; e < B * B; e += 32) aug[(e / B) * 2 * B + B + (e % B)] = d.QQ[ko + e];
    __syncwarp();
    if (!warp_solve<B>(aug, fac, &s_i, M0)) {
      if (lane == 0) d.flag[k] = 2;
      return;
    }
    for (int e = lane; e < B * B; e += 32) M1[e] = d.xi[ko + e];
    __syncwarp();
    warp_matmul<B>(M0, M1, M2);  // alpha xi
    for (int e = lane; e < B * B; e += 32) {
      d.alpha[ko + e] = to32(M0[e]);
      d.axi[ko + e] = to32(M2[e]);
    }
    return;
  }
  // PHASE 0 / 2: Cholesky QR of W
  sum_parts<B>(d, k, 0, M0, B);  // W^H W
  sum_parts<B>(d, k, 1, M1, B);  // W^T W
  if (!warp_cholesky<B>(M0, M2, &s_i)) {  // M2 = Lc, tau = Lc^H
    if (lane == 0) d.flag[k] = 2;
    return;
  }
  warp_lower_inverse<B>(M2, M3);  // M3 = Li = Lc^{-1}, tau^{-1} = Li^H
  // tau^{-1} for the vector kernels: at a restart (PHASE 0) in FP64 for the
  // Q_0 kernel, which writes Q_0 itself into W, so that the FP32 copy is I
  for (int e = lane; e < B * B; e += 32) {
    const int a = e / B, c = e % B;
    const double2 v = M3[c * B + a];
    if (PHASE == 0) {
      d.tinv64[ko + e] = make_double2(v.x, -v.y);
      d.tinv[ko + e] = make_float2(a == c ? 1.f : 0.f, 0.f);
    } else {
      d.tinv[ko + e] = make_float2((float)v.x, (float)-v.y);
    }
  }
  // Q^T Q = tau^{-T} (W^T W) tau^{-1}, with tau^{-1} = Li^H
  {
    // T1 = (W^T W) tau^{-1}, tau^{-1}[m][j] = conj(Li[j][m])
    const int j = lane;
    if (j < B) {
      for (int r = 0; r < B; ++r) {
        double2 v = make_double2(0.0, 0.0);
        for (int m = 0; m < B; ++m) {
          const double2 a = M1[r * B + m];
          const double2 li = M3[j * B + m];
          const double2 b = make_double2(li.x, -li.y);
          v.x += a.x * b.x - a.y * b.y;
          v.y += a.x * b.y + a.y * b.x;
        }
        M0[r * B + j] = v;
      }
    }
    __syncwarp();
    // QQn = tau^{-T} T1, tau^{-T}[a][r] = tau^{-1}[r][a] = conj(Li[a][r])
    if (j < B) {
      for (int a = 0; a < B; ++a) {
        double2 v = make_double2(0.0, 0.0);
        for (int r = 0; r < B; ++r) {
          const double2 li = M3[a * B + r];
          const double2 t = make_double2(li.x, -li.y);
          const double2 b = M0[r * B + j];
          v.x += t.x * b.x - t.y * b.y;
          v.y += t.x * b.y + t.y * b.x;
        }
        M1[a * B + j] = v;  // M1 = Q_{k+1}^T Q_{k+1} (W^T W no longer needed)
      }
    }
    __syncwarp();
  }
  if (PHASE == 0) {
    for (int e = lane; e < B * B; e += 32) {
      const int a = e / B, c = e % B;
      const double2 l = M2[c * B + a];  // tau[a][c] = conj(Lc[c][a])
      d.xi[ko + e] = make_double2(l.x, -l.y);
      d.QQ[ko + e] = M1[e];
    }
    if (lane < B) {
      double s = 0.0;
      for (int a = 0; a < B; ++a) s += cabs2(M2[lane * B + a]);  // column lane of tau = row lane of Lc
      d.xi0n[(size_t)k * B + lane] = sqrt(s);
    }
    if (lane == 0) {
      d.flag[k] = 0;
      d.its[k] = 0;
    }
    return;
  }
  // xi_{k+1} = tau xi_k, tau[a][m] = conj(Lc[m][a]) (m >= a)
  for (int e = lane; e < B * B; e += 32) M0[e] = d.xi[ko + e];
  __syncwarp();
  {
    const int j = lane;
    if (j < B) {
      for (int a = 0; a < B; ++a) {
        double2 v = make_double2(0.0, 0.0);
        for (int m = a; m < B; ++m) {
          const double2 l = M2[m * B + a];
          const double2 t = make_double2(l.x, -l.y);
          const double2 x = M0[m * B + j];
          v.x += t.x * x.x - t.y * x.y;
          v.y += t.x * x.y + t.y * x.x;
        }
        aug[a * 2 * B + B + j] = v;  // staged: tau xi
      }
    }
    __syncwarp();
  }
  for (int e = lane; e < B * B; e += 32) d.xi[ko + e] = aug[(e / B) * 2 * B + B + (e % B)];
  // every column's residual norm ||xi[:, j]|| against its start
  bool conv = true;
  if (lane < B) {
    double s = 0.0;
    for (int a = 0; a < B; ++a) s += cabs2(aug[a * 2 * B + B + lane]);
    conv = sqrt(s) <= d.tol_in * d.xi0n[(size_t)k * B + lane];
  }
  conv = __all_sync(0xffffffffu, conv);
  __syncwarp();
  // beta = QQ_k^{-1} (tau^T QQ_{k+1}); tau^T[a][m] = tau[m][a] = conj(Lc[a][m]) (m <= a)
  {
    const int j = lane;
    if (j < B) {
      for (int a = 0; a < B; ++a) {
        double2 v = make_double2(0.0, 0.0);
        for (int m = 0; m <= a; ++m) {
          const double2 l = M2[a * B + m];
          const double2 t = make_double2(l.x, -l.y);
          const double2 q = M1[m * B + j];
          v.x += t.x * q.x - t.y * q.y;
          v.y += t.x * q.y + t.y * q.x;
        }
        aug[a * 2 * B + B + j] = v;
      }
    }
    __syncwarp();
  }
  for (int e = lane; e < B * B; e += 32) aug[(e / B) * 2 * B + (e % B)] = d.QQ[ko + e];
  __syncwarp();
  const bool ok = warp_solve<B>(aug, fac, &s_i, M0);  // M0 = beta
  for (int e = lane; e < B * B; e += 32) {
    d.QQ[ko + e] = M1[e];
    if (ok) d.beta[ko + e] = to32(M0[e]);
  }
  if (lane == 0) {
    const int it = d.its[k] + 1;
    d.its[k] = it;
    d.flag[k] = conv ? 1 : !ok ? 2 : it >= d.icap[k] ? 3 : 0;
  }
}

// ---------------------------------------------------------------------------
// Outer (FP64) steps over the members of the listed blocks: grid.y = listed
// blocks x B, member v = blist[y / B] * B + y % B.
// ---------------------------------------------------------------------------
// R = e_col - A X (A X already in R when have_ax), partial ||R||^2 and
// sum_{i} Gamma_L(i) |X(i)|^2 per chunk of points.
__global__ void __launch_bounds__(kBlkThreads) blk_resid_kernel(const BlkDev* __restrict__ dp, int have_ax) {
  const BlkDev& d = *dp;
  const int B = d.B;
  const int v = d.blist[blockIdx.y / B] * B + (int)(blockIdx.y % B);
  const long long N = d.N;
  const long long x0 = (long long)blockIdx.x * d.chunkR_pts;
  const long long x1 = min(N, x0 + d.chunkR_pts);
  const int col = d.col[v];
  double2* R = d.R + (size_t)v * N;
  const double2* X = d.X + (size_t)v * N;
  double acc[2] = {0.0, 0.0};
  for (long long i = x0 + threadIdx.x; i < x1; i += blockDim.x) {
    double2 r = have_ax ? R[i] : make_double2(0.0, 0.0);
    r.x = (i == col ? 1.0 : 0.0) - r.x;
    r.y = -r.y;
    R[i] = r;
    acc[0] += cabs2(r);
    const double g = d.gl[i];
    if (g > 0.0) acc[1] += g * cabs2(X[i]);
  }
  __shared__ double red[32 * 2];
  double out[2];
  block_sum<2>(acc, red, out);
  if (threadIdx.x == 0) {
    double* p = d.rpart + ((size_t)v * d.nchunkR + blockIdx.x) * 2;
    p[0] = out[0];
    p[1] = out[1];
  }
}

// rn = ||R||, tt = sum Gamma_L |X|^2 per listed member (chunks in order)
__global__ void blk_norm_kernel(const BlkDev* __restrict__ dp, int n_members) {
  const BlkDev& d = *dp;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= n_members) return;
  const int B = d.B;
  const int v = d.blist[y / B] * B + y % B;
  double s0 = 0.0, s1 = 0.0;
  for (int ch = 0; ch < d.nchunkR; ++ch) {
    s0 += d.rpart[((size_t)v * d.nchunkR + ch) * 2];
    s1 += d.rpart[((size_t)v * d.nchunkR + ch) * 2 + 1];
  }
  d.rn[v] = sqrt(s0);
  d.tt[v] = s1;
}

// R <- R / ||R|| per member (FP64, in place): the right-hand sides of the next
// inner solve, each of unit norm
__global__ void __launch_bounds__(kBlkThreads) blk_scale_kernel(const BlkDev* __restrict__ dp) {
  const BlkDev& d = *dp;
  const int B = d.B;
  const int v = d.blist[blockIdx.y / B] * B + (int)(blockIdx.y % B);
  const long long N = d.N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double rn = d.rn[v];
  const double s = rn > 0.0 ? 1.0 / rn : 0.0;
  double2 r = d.R[(size_t)v * N + i];
  r.x *= s;
  r.y *= s;
  d.R[(size_t)v * N + i] = r;
}

// X += ||R|| D (the inner solution solves A D = R / ||R|| per column)
__global__ void __launch_bounds__(kBlkThreads) blk_xupd_kernel(const BlkDev* __restrict__ dp) {
  const BlkDev& d = *dp;
  const int B = d.B;
  const int v = d.blist[blockIdx.y / B] * B + (int)(blockIdx.y % B);
  const long long N = d.N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double rn = d.rn[v];
  const float2 dd = d.D[(size_t)v * N + i];
  double2 x = d.X[(size_t)v * N + i];
  x.x = fma(rn, (double)dd.x, x.x);
  x.y = fma(rn, (double)dd.y, x.y);
  d.X[(size_t)v * N + i] = x;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define RSN_BLK_DISPATCH(B, CALL) \
  switch (B) {                    \
    case 4: CALL(4); break;       \
    case 8: CALL(8); break;       \
    case 16: CALL(16); break;     \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_blk_comb_p(int B, int nb, cudaStream_t st, const BlkDev* d, long long N) {
  const dim3 grid((unsigned)((N + kBlkThreads - 1) / kBlkThreads), nb);
#define L_(BB) blk_comb_p_kernel<BB><<<grid, kBlkThreads, 0, st>>>(d)
  RSN_BLK_DISPATCH(B, L_)
#undef L_
  return cudaGetLastError();
}

cudaError_t launch_blk_comb_w(int B, int nb, cudaStream_t st, const BlkDev* d, long long N) {
  const dim3 grid((unsigned)((N + kBlkThreads - 1) / kBlkThreads), nb);
#define L_(BB) blk_comb_w_kernel<BB><<<grid, kBlkThreads, 0, st>>>(d)
  RSN_BLK_DISPATCH(B, L_)
#undef L_
  return cudaGetLastError();
}

cudaError_t launch_blk_gram(int B, int mode, int nb, int nchunk, cudaStream_t st, const BlkDev* d) {
  const dim3 grid(nchunk, nb);
  if (mode == 0) {
#define L_(BB) blk_gram_kernel<BB, 0><<<grid, kBlkThreads, 0, st>>>(d)
    RSN_BLK_DISPATCH(B, L_)
#undef L_
  } else {
#define L_(BB) blk_gram_kernel<BB, 1><<<grid, kBlkThreads, 0, st>>>(d)
    RSN_BLK_DISPATCH(B, L_)
#undef L_
  }
  return cudaGetLastError();
}

cudaError_t launch_blk_gram64(int B, int nb, int nchunk, cudaStream_t st, const BlkDev* d) {
  const dim3 grid(nchunk, nb);
#define L_(BB) blk_gram64_kernel<BB><<<grid, kBlkThreads, 0, st>>>(d)
  RSN_BLK_DISPATCH(B, L_)
#undef L_
  return cudaGetLastError();
}

cudaError_t launch_blk_q0(int B, int nb, cudaStream_t st, const BlkDev* d, long long N) {
  const dim3 grid((unsigned)((N + kBlkThreads - 1) / kBlkThreads), nb);
#define L_(BB) blk_q0_kernel<BB><<<grid, kBlkThreads, 0, st>>>(d)
  RSN_BLK_DISPATCH(B, L_)
#undef L_
  return cudaGetLastError();
}

cudaError_t launch_blk_small(int B, int phase, int nb, cudaStream_t st, const BlkDev* d) {
  if (phase == 0) {
#define L_(BB) blk_small_kernel<BB, 0><<<nb, 32, 0, st>>>(d)
    RSN_BLK_DISPATCH(B, L_)
#undef L_
  } else if (phase == 1) {
#define L_(BB) blk_small_kernel<BB, 1><<<nb, 32, 0, st>>>(d)
    RSN_BLK_DISPATCH(B, L_)
#undef L_
  } else {
#define L_(BB) blk_small_kernel<BB, 2><<<nb, 32, 0, st>>>(d)
    RSN_BLK_DISPATCH(B, L_)
#undef L_
  }
  return cudaGetLastError();
}

cudaError_t launch_blk_resid(int B, int nb, int nchunkR, bool have_ax, cudaStream_t st, const BlkDev* d) {
  blk_resid_kernel<<<dim3(nchunkR, nb * B), kBlkThreads, 0, st>>>(d, have_ax ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_blk_norm(int B, int nb, int nchunkR, cudaStream_t st, const BlkDev* d) {
  (void)nchunkR;
  const int n = nb * B;
  blk_norm_kernel<<<(n + 127) / 128, 128, 0, st>>>(d, n);
  return cudaGetLastError();
}

cudaError_t launch_blk_scale(int B, int nb, cudaStream_t st, const BlkDev* d, long long N) {
  blk_scale_kernel<<<dim3((unsigned)((N + kBlkThreads - 1) / kBlkThreads), nb * B), kBlkThreads, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_blk_xupd(int B, int nb, cudaStream_t st, const BlkDev* d, long long N) {
  blk_xupd_kernel<<<dim3((unsigned)((N + kBlkThreads - 1) / kBlkThreads), nb * B), kBlkThreads, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace rsn
