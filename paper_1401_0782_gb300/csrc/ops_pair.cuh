// FP32 operator kernel on point pairs with plane streaming: y = A_loc(E) v
// (COCG) or y = A(E) x (apply), A(E) = E - H_KS + i(Gamma_L + Gamma_R) (Eqs. G
// and Hop), H_KS = -1/2 lap_FD + V_loc [+ sum_p |v_p> e_kb <v_p| in the apply
// mode] (Sec. II.C).
//
// One CTA owns whole x-y planes [z0, z0+Lz) of one slot and marches along z.
//  * The input planes (r and p_old, or x) of planes z0-R .. z0+Lz+R-1 arrive by
//    bulk copies (TMA, cp.async.bulk) in a ring of kPairStages shared-memory
//    stages, issued kPairStages planes ahead of use and completed on one
//    mbarrier per stage, so the bytes in flight cost no registers.
//  * Each thread owns two x-neighbours (x0, x0+1) of one row (nx even), so each
//    shared-memory access moves one 128-bit pair and each global store 16 bytes.
//  * The 2R+1 produced planes around the current one sit in a register ring
//    whose slot for plane z is (z - z0 + R) mod (2R+1); the march is unrolled by
//    2R+1, so every ring index is a compile-time constant and nothing is shifted.
//  * The current plane goes through a double-buffered shared-memory tile for
//    the x and y neighbours (one barrier per plane), whose row pitch nx + 16 lets
//    a quarter warp that crosses a row boundary still touch 32 distinct banks;
//    the zero columns and rows around it are the Dirichlet boundary.
//
// FP32 accuracy: the neighbour terms at distances m <= 2, whose weights carry
// the large part of the Laplacian, are summed in difference form,
// w_m sum_nb (v_nb - v_c): near-equal values subtract exactly, so the large
// FD diagonal never meets the small result of smooth fields.  The terms at
// m > 2 (weights below 1/10 of w_1) are summed directly, and their share of
// the diagonal, -6 sum_{m>2} w_m, is folded into E - V_loc.
#pragma once
#include "cplx.cuh"
#include "rsn_internal.h"
#include "tma.cuh"

namespace rsn {

// elementwise a + b, a - b, a * b + c on (re, im) pairs (the compiler pairs
// them into Blackwell's two-wide FP32 instructions where that pays; explicit
// f32x2 inline assembly measured slower, its operand packing costs moves)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
// acc + a * b for complex a, b
__device__ __forceinline__ float2 cfma2(float2 a, float2 b, float2 acc) {
  acc = fma2(make_float2(a.x, a.x), b, acc);
  return fma2(make_float2(-a.y, a.y), make_float2(b.y, b.x), acc);
}

// Kahan-compensated accumulation (sum, carry) for long FP32 dot products.
__device__ __forceinline__ void kahan_add_f(float& sum, float& carry, float term) {
  const float y = term - carry;
  const float t = sum + y;
  carry = (t - sum) - y;
  sum = t;
}

struct Pair {
  float2 a, b;  // values at x0 and x0 + 1
};

__device__ __forceinline__ Pair zero_pair() { return Pair{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

__device__ __forceinline__ Pair lds_pair(const float2* s) {
  const float4 v = *reinterpret_cast<const float4*>(s);
  return Pair{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void sts_pair(float2* s, const Pair& v) {
  *reinterpret_cast<float4*>(s) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}


template <int R, int MODE, bool BIG>
__global__ void __maxnreg__(96)
op_pair_kernel(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp, const void* __restrict__ x_in,
               void* __restrict__ y_out, const void* __restrict__ c_in) {
  constexpr int Q = 2 * R + 1;
  constexpr int MD = R < 2 ? R : 2;  // distances summed in difference form
  constexpr int KX = (R + 1) / 2;    // neighbour pairs left / right in x
  constexpr int NIN = (MODE == OP_COCG) ? 2 : 1;
  const BatchDev& b = *bp;
  const int s = blockIdx.y;
  if constexpr (MODE == OP_COCG) {
    if (b.state[s] != SL_ACTIVE) return;
  }
  const JuncDev& J = jt[b.junc[s]];
  const int tile = blockIdx.x;
  if (tile >= J.nA || J.kind != kOpPair) return;

  const int nx = J.nx, ny = J.ny, nz = J.nz, plane = J.plane;
  const int hx = nx >> 1;  // pairs per row
  const int z0 = tile * J.Lz, z1 = min(z0 + J.Lz, nz);
  const int pitch = nx + 2 * kPairXO;
  const int rows = ny + 2 * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long vo = b.voff[s];
  const int n_proj = J.n_proj;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* stage = reinterpret_cast<float2*>(smem_raw);  // [kPairStages][NIN][plane]
  float2* exch = stage + kPairStages * NIN * plane;    // [2][rows][pitch]
  float2* ce = exch + 2 * rows * pitch;                 // apply mode: e_kb[p] (v_p . x)
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(ce + (MODE == OP_APPLY ? n_proj + kCePad : 0)) + 15) &
      ~static_cast<uintptr_t>(15));
  __shared__ double red[32 * 2];
  __shared__ int s_bad;

  for (int i = tid; i < 2 * rows * pitch; i += nt) exch[i] = make_float2(0.f, 0.f);
  if (tid == 0) {
    for (int k = 0; k < kPairStages; ++k) mbar_init(bars + k, 1);
    s_bad = 0;
  }

  // ---- per-system scalars and vectors --------------------------------------
  const int k = (MODE == OP_COCG) ? b.iters[s] : 0;
  const bool first = (MODE == OP_COCG) && (k == 0);
  float2 beta = make_float2(0.f, 0.f);
  if (MODE == OP_COCG && !first) beta = make_float2((float)b.beta_cur[s].x, (float)b.beta_cur[s].y);
  const float2* src0;
  const float2* src1 = nullptr;
  float2* pnew = nullptr;
  float2* yv;
  if constexpr (MODE == OP_COCG) {
    src0 = reinterpret_cast<const float2*>(b.r) + vo;
    if (!first) src1 = reinterpret_cast<const float2*>((k & 1) ? b.p1 : b.p0) + vo;
    pnew = reinterpret_cast<float2*>((k & 1) ? b.p0 : b.p1) + vo;
    yv = reinterpret_cast<float2*>(b.q) + vo;
  } else {
    src0 = reinterpret_cast<const float2*>(x_in) + vo;
    yv = reinterpret_cast<float2*>(y_out) + vo;
  }
  if (MODE == OP_APPLY && n_proj > 0) {
    const float2* cin = reinterpret_cast<const float2*>(c_in) + (size_t)s * b.pstride;
    for (int p = tid; p < n_proj; p += nt) {
      const float e = (float)J.ekb[p];
      const float2 c = cin[p];
      ce[p] = make_float2(e * c.x, e * c.y);
    }
    for (int p = tid; p < kCePad; p += nt) ce[n_proj + p] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  // planes [zb, ze) stream through the ring; plane zl uses stage (zl - zb) % kPairStages
  const int zb = z0 - R, ze = z1 + R;
  const uint32_t pbytes = (uint32_t)(plane * sizeof(float2));
  auto issue = [&](int zl) {
    const int st = (zl - zb) % kPairStages;
    uint64_t* bar = bars + st;
    if (zl >= 0 && zl < nz) {
      mbar_arrive_expect_tx(bar, src1 ? 2 * pbytes : pbytes);
      bulk_g2s(stage + (st * NIN) * plane, src0 + (size_t)zl * plane, pbytes, bar);
      if (src1) bulk_g2s(stage + (st * NIN + 1) * plane, src1 + (size_t)zl * plane, pbytes, bar);
    } else {
      mbar_arrive(bar);  // nothing to copy outside the box: complete the phase
    }
  };
  if (tid == 0) {
    fence_proxy_async();
    for (int f = 0; f < kPairStages && zb + f < ze; ++f) issue(zb + f);
  }

  // ---- owned pair ------------------------------------------------------------
  const bool own = tid < ny * hx;
  const int yl = own ? tid / hx : 0;
  const int x0 = own ? 2 * (tid - yl * hx) : 0;
  const int po = x0 + yl * nx;                     // offset within a plane (even)
  const int so = (yl + R) * pitch + x0 + kPairXO;  // exchange-tile index of the pair (even)

  // FD weights and E - 6 sum_{m > MD} w_m (the direct terms' share of the
  // diagonal) in shared memory: broadcast reads instead of live registers
  __shared__ float s_w[R + 2];
  if (tid == 0) {
    float dshift = 0.f;
    for (int m = 1; m <= R; ++m) {
      s_w[m] = J.w32[m];
      if (m > MD) dshift -= 6.f * J.w32[m];
    }
    s_w[0] = (float)b.E[s] + dshift;
  }
  __syncthreads();
  const float4* dg4 = reinterpret_cast<const float4*>(J.dg32);
  float4 dgn = make_float4(0.f, 0.f, 0.f, 0.f);  // (-V_loc, Gamma) of both points of the next plane
  if (own && z0 < z1) dgn = __ldg(dg4 + ((z0 * plane + po) >> 1));

  Pair zq[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) zq[m] = zero_pair();
  float2 macc = make_float2(0.f, 0.f), mcar = macc;  // Kahan sum of mu = v^T A_loc v
  int sidx = 0;                                      // stage of the plane entering the ring
  uint32_t sph = 0;                                  // its mbarrier phase parity

  for (int zr = z0 - 2 * R; zr < z1; zr += Q) {
#pragma unroll
    for (int u = 0; u < Q; ++u) {
      const int zc = zr + u;
      if (zc < z1) {
        // plane zl = zc + R arrives in stage sidx and enters ring slot u
        const int zl = zc + R;
        Pair v = zero_pair();
        if (!mbar_wait(bars + sidx, sph)) {
          s_bad = 1;
        } else if (own && zl >= 0 && zl < nz) {
          v = lds_pair(stage + (sidx * NIN) * plane + po);
          if constexpr (MODE == OP_COCG) {
            if (src1) {
              const Pair pp = lds_pair(stage + (sidx * NIN + 1) * plane + po);
              v.a = cfma2(beta, pp.a, v.a);
              v.b = cfma2(beta, pp.b, v.b);
            }
          }
        }
        zq[u] = v;
        const int C = (u + R + 1) % Q;  // ring slot of plane zc (a constant once unrolled)
        float2* smb = exch + (((zc - z0) & 1) ? rows * pitch : 0);
        if (zc >= z0 && own) sts_pair(smb + so, zq[C]);
        __syncthreads();
        if (s_bad) {
          // a copy never arrived: report, let in-flight copies land (bounded), leave
          if (tid == 0) {
            if (b.sched) atomicExch(b.sched + 2, 1);
            for (int f = 0; f < kPairStages; ++f) {
              const int zq2 = zl + f;
              if (zq2 < ze) mbar_wait(bars + (zq2 - zb) % kPairStages, (uint32_t)(((zq2 - zb) / kPairStages) & 1));
            }
          }
          return;
        }
        // every thread has read stage sidx: refill it with plane zl + kPairStages
        if (tid == 0 && zl + kPairStages < ze) {
          fence_proxy_async();
          issue(zl + kPairStages);
        }
        if (++sidx == kPairStages) {
          sidx = 0;
          sph ^= 1u;
        }
        if (zc >= z0 && own) {
          const float4 dgc = dgn;
          if (zc + 1 < z1) dgn = __ldg(dg4 + (((zc + 1) * plane + po) >> 1));
          // x neighbours at offsets -2KX .. 2KX+1 from x0
          float2 X[4 * KX + 2];
#pragma unroll
          for (int kk = 0; kk < 2 * KX + 1; ++kk) {
            const Pair pr = (kk == KX) ? zq[C] : lds_pair(smb + so + 2 * (kk - KX));
            X[2 * kk] = pr.a;
            X[2 * kk + 1] = pr.b;
          }
          float2 lap0 = make_float2(0.f, 0.f), lap1 = lap0;
          const float2 c0 = zq[C].a, c1 = zq[C].b;
#pragma unroll
          for (int m = 1; m <= R; ++m) {
            const Pair zm = zq[(C + Q - m) % Q], zp = zq[(C + m) % Q];
            const Pair ym = lds_pair(smb + so - m * pitch), yp = lds_pair(smb + so + m * pitch);
            const float2 xm0 = X[2 * KX - m], xp0 = X[2 * KX + m];
            const float2 xm1 = X[2 * KX + 1 - m], xp1 = X[2 * KX + 1 + m];
            const float2 w = make_float2(s_w[m], s_w[m]);
            float2 s0, s1;
            if (m <= MD) {
              s0 = add2(add2(add2(sub2(zm.a, c0), sub2(zp.a, c0)), add2(sub2(ym.a, c0), sub2(yp.a, c0))),
                        add2(sub2(xm0, c0), sub2(xp0, c0)));
              s1 = add2(add2(add2(sub2(zm.b, c1), sub2(zp.b, c1)), add2(sub2(ym.b, c1), sub2(yp.b, c1))),
                        add2(sub2(xm1, c1), sub2(xp1, c1)));
            } else {
              s0 = add2(add2(add2(zm.a, zp.a), add2(ym.a, yp.a)), add2(xm0, xp0));
              s1 = add2(add2(add2(zm.b, zp.b), add2(ym.b, yp.b)), add2(xm1, xp1));
            }
            lap0 = fma2(w, s0, lap0);
            lap1 = fma2(w, s1, lap1);
          }
          // + (E - V_loc + dshift + i Gamma) v
          const float Ef = s_w[0];
          float2 y0v = cfma2(make_float2(Ef + dgc.x, dgc.y), c0, lap0);
          float2 y1v = cfma2(make_float2(Ef + dgc.z, dgc.w), c1, lap1);
          const int gi = zc * plane + po;
          if constexpr (MODE == OP_APPLY) {
            if (n_proj > 0) {
              const int nq = J.inv_nq;
#pragma unroll
              for (int jj = 0; jj < 2; ++jj) {
                float2 yy = jj ? y1v : y0v;
                const int e0 = J.inv_ptr[gi + jj], e1 = J.inv_ptr[gi + jj + 1];
                for (int e = e0; e < e1; ++e) {
                  const float2* cp = ce + J.inv_p0[e];
                  for (int qd = 0; qd < nq; ++qd) {
                    const float4 a = J.inv_q32[e * nq + qd];
                    yy = fma2(make_float2(-a.x, -a.x), cp[4 * qd], yy);
                    yy = fma2(make_float2(-a.y, -a.y), cp[4 * qd + 1], yy);
                    yy = fma2(make_float2(-a.z, -a.z), cp[4 * qd + 2], yy);
                    yy = fma2(make_float2(-a.w, -a.w), cp[4 * qd + 3], yy);
                  }
                }
                if (jj) y1v = yy;
                else y0v = yy;
              }
            }
          }
          if constexpr (MODE == OP_COCG) {
            *reinterpret_cast<float4*>(pnew + gi) = make_float4(c0.x, c0.y, c1.x, c1.y);
            // mu partial v^T y (unconjugated) of both points, Kahan-compensated
            float2 t = fma2(make_float2(c0.x, c0.x), y0v, make_float2(0.f, 0.f));
            t = fma2(make_float2(-c0.y, c0.y), make_float2(y0v.y, y0v.x), t);
            t = fma2(make_float2(c1.x, c1.x), y1v, t);
            t = fma2(make_float2(-c1.y, c1.y), make_float2(y1v.y, y1v.x), t);
            const float2 yk = sub2(t, mcar);
            const float2 tk = add2(macc, yk);
            mcar = sub2(sub2(tk, macc), yk);
            macc = tk;
          }
          *reinterpret_cast<float4*>(yv + gi) = make_float4(y0v.x, y0v.y, y1v.x, y1v.y);
        }
      }
    }
  }
  if constexpr (MODE == OP_COCG) {
    float vv[2] = {macc.x - mcar.x, macc.y - mcar.y};
    double out[2];
    block_sum<2>(vv, red, out);
    if (tid == 0) b.mu_part[(size_t)s * b.PA + tile] = make_double2(out[0], out[1]);
  }
}

// ---------------------------------------------------------------------------
// One point per thread, whole planes streamed by bulk copies: the same march
// as op_pair_kernel (bulk-copied input planes, register ring of 2R+1 produced
// planes unrolled by 2R+1, double-buffered exchange tile, hybrid difference
// form) with one grid point per thread, so that the z ring takes 2R+1 complex
// values and two CTAs of up to kPlaneThreads threads fit one SM.  Any nx; the
// plane size must be even (16-byte bulk copies).
// ---------------------------------------------------------------------------
template <int R, int MODE>
__global__ void __launch_bounds__(kPlaneThreads, 2)
op_plane_kernel(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp, const void* __restrict__ x_in,
                void* __restrict__ y_out, const void* __restrict__ c_in) {
  constexpr int Q = 2 * R + 1;
  constexpr int MD = R < 2 ? R : 2;  // distances summed in difference form
  constexpr int NIN = (MODE == OP_COCG) ? 2 : 1;
  const BatchDev& b = *bp;
  const int s = blockIdx.y;
  if constexpr (MODE == OP_COCG) {
    if (b.state[s] != SL_ACTIVE) return;
  }
  const JuncDev& J = jt[b.junc[s]];
  const int tile = blockIdx.x;
  if (tile >= J.nA || J.kind != kOpPlane) return;

  const int nx = J.nx, ny = J.ny, nz = J.nz, plane = J.plane;
  const int z0 = tile * J.Lz, z1 = min(z0 + J.Lz, nz);
  const int pitch = nx + 2 * kPairXO;
  const int rows = ny + 2 * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long vo = b.voff[s];
  const int n_proj = J.n_proj;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* stage = reinterpret_cast<float2*>(smem_raw);  // [kPairStages][NIN][plane]
  float2* exch = stage + kPairStages * NIN * plane;    // [2][rows][pitch]
  float2* ce = exch + 2 * rows * pitch;                 // apply mode: e_kb[p] (v_p . x)
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(ce + (MODE == OP_APPLY ? n_proj + kCePad : 0)) + 15) &
      ~static_cast<uintptr_t>(15));
  __shared__ double red[32 * 2];
  __shared__ int s_bad;
  __shared__ float s_w[R + 2];

  for (int i = tid; i < 2 * rows * pitch; i += nt) exch[i] = make_float2(0.f, 0.f);
  if (tid == 0) {
    for (int k = 0; k < kPairStages; ++k) mbar_init(bars + k, 1);
    s_bad = 0;
    // FD weights and E - 6 sum_{m > MD} w_m (the direct terms' share of the diagonal)
    float dshift = 0.f;
    for (int m = 1; m <= R; ++m) {
      s_w[m] = J.w32[m];
      if (m > MD) dshift -= 6.f * J.w32[m];
    }
    s_w[0] = (float)b.E[s] + dshift;
  }

  const int k = (MODE == OP_COCG) ? b.iters[s] : 0;
  const bool first = (MODE == OP_COCG) && (k == 0);
  float2 beta = make_float2(0.f, 0.f);
  if (MODE == OP_COCG && !first) beta = make_float2((float)b.beta_cur[s].x, (float)b.beta_cur[s].y);
  const float2* src0;
  const float2* src1 = nullptr;
  float2* pnew = nullptr;
  float2* yv;
  if constexpr (MODE == OP_COCG) {
    src0 = reinterpret_cast<const float2*>(b.r) + vo;
    if (!first) src1 = reinterpret_cast<const float2*>((k & 1) ? b.p1 : b.p0) + vo;
    pnew = reinterpret_cast<float2*>((k & 1) ? b.p0 : b.p1) + vo;
    yv = reinterpret_cast<float2*>(b.q) + vo;
  } else {
    src0 = reinterpret_cast<const float2*>(x_in) + vo;
    yv = reinterpret_cast<float2*>(y_out) + vo;
  }
  if (MODE == OP_APPLY && n_proj > 0) {
    const float2* cin = reinterpret_cast<const float2*>(c_in) + (size_t)s * b.pstride;
    for (int p = tid; p < n_proj; p += nt) {
      const float e = (float)J.ekb[p];
      const float2 c = cin[p];
      ce[p] = make_float2(e * c.x, e * c.y);
    }
    for (int p = tid; p < kCePad; p += nt) ce[n_proj + p] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  const int zb = z0 - R, ze = z1 + R;
  const uint32_t pbytes = (uint32_t)(plane * sizeof(float2));
  auto issue = [&](int zl) {
    const int st = (zl - zb) % kPairStages;
    uint64_t* bar = bars + st;
    if (zl >= 0 && zl < nz) {
      mbar_arrive_expect_tx(bar, src1 ? 2 * pbytes : pbytes);
      bulk_g2s(stage + (st * NIN) * plane, src0 + (size_t)zl * plane, pbytes, bar);
      if (src1) bulk_g2s(stage + (st * NIN + 1) * plane, src1 + (size_t)zl * plane, pbytes, bar);
    } else {
      mbar_arrive(bar);
    }
  };
  if (tid == 0) {
    fence_proxy_async();
    for (int f = 0; f < kPairStages && zb + f < ze; ++f) issue(zb + f);
  }

  const bool own = tid < plane;
  const int yl = own ? tid / nx : 0;
  const int xl = own ? tid - yl * nx : 0;
  const int so = (yl + R) * pitch + xl + kPairXO;  // exchange-tile index of the point

  float2 dgn = make_float2(0.f, 0.f);  // (-V_loc, Gamma) of the next plane to compute
  if (own && z0 < z1) dgn = __ldg(J.dg32 + (z0 * plane + tid));

  float2 zq[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) zq[m] = make_float2(0.f, 0.f);
  float ma_x = 0.f, ma_y = 0.f, mc_x = 0.f, mc_y = 0.f;  // Kahan sum of mu = v^T A_loc v
  int sidx = 0;
  uint32_t sph = 0;

  for (int zr = z0 - 2 * R; zr < z1; zr += Q) {
#pragma unroll
    for (int u = 0; u < Q; ++u) {
      const int zc = zr + u;
      if (zc < z1) {
        const int zl = zc + R;
        float2 v = make_float2(0.f, 0.f);
        if (!mbar_wait(bars + sidx, sph)) {
          s_bad = 1;
        } else if (own && zl >= 0 && zl < nz) {
          v = stage[(sidx * NIN) * plane + tid];
          if constexpr (MODE == OP_COCG) {
            if (src1) {
              const float2 pp = stage[(sidx * NIN + 1) * plane + tid];
              v.x = fmaf(beta.x, pp.x, fmaf(-beta.y, pp.y, v.x));
              v.y = fmaf(beta.x, pp.y, fmaf(beta.y, pp.x, v.y));
            }
          }
        }
        zq[u] = v;
        const int C = (u + R + 1) % Q;  // ring slot of plane zc (a constant once unrolled)
        float2* smb = exch + (((zc - z0) & 1) ? rows * pitch : 0);
        if (zc >= z0 && own) smb[so] = zq[C];
        __syncthreads();
        if (s_bad) {
          if (tid == 0) {
            if (b.sched) atomicExch(b.sched + 2, 1);
            for (int f = 0; f < kPairStages; ++f) {
              const int zq2 = zl + f;
              if (zq2 < ze) mbar_wait(bars + (zq2 - zb) % kPairStages, (uint32_t)(((zq2 - zb) / kPairStages) & 1));
            }
          }
          return;
        }
        if (tid == 0 && zl + kPairStages < ze) {
          fence_proxy_async();
          issue(zl + kPairStages);
        }
        if (++sidx == kPairStages) {
          sidx = 0;
          sph ^= 1u;
        }
        if (zc >= z0 && own) {
          const float2 dgc = dgn;
          if (zc + 1 < z1) dgn = __ldg(J.dg32 + ((zc + 1) * plane + tid));
          const float2 c = zq[C];
          float lx = 0.f, ly = 0.f;
#pragma unroll
          for (int m = 1; m <= R; ++m) {
            const float2 zm = zq[(C + Q - m) % Q], zp = zq[(C + m) % Q];
            const float2 ym = smb[so - m * pitch], yp = smb[so + m * pitch];
            const float2 xm = smb[so - m], xp = smb[so + m];
            const float w = s_w[m];
            float sx, sy;
            if (m <= MD) {
              sx = ((zm.x - c.x) + (zp.x - c.x)) + ((ym.x - c.x) + (yp.x - c.x)) + ((xm.x - c.x) + (xp.x - c.x));
              sy = ((zm.y - c.y) + (zp.y - c.y)) + ((ym.y - c.y) + (yp.y - c.y)) + ((xm.y - c.y) + (xp.y - c.y));
            } else {
              sx = ((zm.x + zp.x) + (ym.x + yp.x)) + (xm.x + xp.x);
              sy = ((zm.y + zp.y) + (ym.y + yp.y)) + (xm.y + xp.y);
            }
            lx = fmaf(w, sx, lx);
            ly = fmaf(w, sy, ly);
          }
          // + (E - V_loc + dshift + i Gamma) v
          const float dr = s_w[0] + dgc.x, di = dgc.y;
          float2 y = make_float2(fmaf(dr, c.x, fmaf(-di, c.y, lx)), fmaf(dr, c.y, fmaf(di, c.x, ly)));
          const int gi = zc * plane + tid;
          if constexpr (MODE == OP_APPLY) {
            if (n_proj > 0) {
              const int nq = J.inv_nq;
              const int e0 = J.inv_ptr[gi], e1 = J.inv_ptr[gi + 1];
              for (int e = e0; e < e1; ++e) {
                const float2* cp = ce + J.inv_p0[e];
                for (int qd = 0; qd < nq; ++qd) {
                  const float4 a = J.inv_q32[e * nq + qd];
                  const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                  for (int jj = 0; jj < 4; ++jj) {
                    y.x = fmaf(-av[jj], cp[4 * qd + jj].x, y.x);
                    y.y = fmaf(-av[jj], cp[4 * qd + jj].y, y.y);
                  }
                }
              }
            }
          }
          if constexpr (MODE == OP_COCG) {
            pnew[gi] = c;
            // mu partial v^T y (unconjugated), Kahan-compensated
            kahan_add_f(ma_x, mc_x, fmaf(c.x, y.x, -c.y * y.y));
            kahan_add_f(ma_y, mc_y, fmaf(c.x, y.y, c.y * y.x));
          }
          yv[gi] = y;
        }
      }
    }
  }
  if constexpr (MODE == OP_COCG) {
    float vv[2] = {ma_x - mc_x, ma_y - mc_y};
    double out[2];
    block_sum<2>(vv, red, out);
    if (tid == 0) b.mu_part[(size_t)s * b.PA + tile] = make_double2(out[0], out[1]);
  }
}

template <int R>
cudaError_t launch_op_plane_r(int mode, dim3 grid, int threads, size_t smem, cudaStream_t st, const JuncDev* jt,
                              const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  void (*kern)(const JuncDev*, const BatchDev*, const void*, void*, const void*) = nullptr;
  if (mode == OP_COCG) kern = op_plane_kernel<R, OP_COCG>;
  else if (mode == OP_APPLY) kern = op_plane_kernel<R, OP_APPLY>;
  else return cudaErrorInvalidValue;
  if (threads > kPlaneThreads) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  kern<<<grid, threads, smem, st>>>(jt, b, x_in, y_out, c_in);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_op_pair_r(int mode, bool big, dim3 grid, int threads, size_t smem, cudaStream_t st,
                             const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  void (*kern)(const JuncDev*, const BatchDev*, const void*, void*, const void*) = nullptr;
  if (mode == OP_COCG) kern = big ? op_pair_kernel<R, OP_COCG, true> : op_pair_kernel<R, OP_COCG, false>;
  else if (mode == OP_APPLY) kern = big ? op_pair_kernel<R, OP_APPLY, true> : op_pair_kernel<R, OP_APPLY, false>;
  else return cudaErrorInvalidValue;
  if (threads > (big ? kPairThreadsBig : kPairThreads)) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  kern<<<grid, threads, smem, st>>>(jt, b, x_in, y_out, c_in);
  return cudaGetLastError();
}

}  // namespace rsn
