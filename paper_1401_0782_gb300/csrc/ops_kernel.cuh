// Operator kernel: y = A(E) v with A(E) = E - H_KS + i(Gamma_L + Gamma_R)
// (Eqs. G and Hop), H_KS = -1/2 lap_FD + V_loc + sum_p |v_p> e_kb <v_p| (Sec. II.C).
//
// One CTA owns a tile of full x rows (y rows [y0, y0+TY)) and z planes
// [z0, z0+Lz) of one slot, and marches along z.  Each thread owns PPT (x, y)
// columns of the tile and keeps the 2R+1 planes around the current one in
// registers, so z neighbours are never re-read; loads run PF planes ahead of
// their use to keep enough bytes in flight.  The current plane (plus R halo
// rows above and below, zero outside the box) is exchanged through a
// double-buffered shared-memory tile for the x and y neighbours: one barrier
// per plane.  Every vector element is read from memory once per tile (plus
// 2R halo planes per z chunk and the halo rows of y tiles).
//
// The value fed to the stencil is produced on the fly, which fuses the
// neighbouring vector update into the matvec:
//   OP_COCG : v = r + beta p_old   (COCG direction update), writes p_new = v,
//             q = A_loc v (A without the projector term) and the partial sums
//             of mu = v^T A v (unconjugated); the projector term of A v is
//             added to q by the update kernel, its share of mu comes from the
//             projections (-sum_p e_kb[p] c_p^2).
//   OP_RESID: v = x64 + d          (refinement iterate), writes r = b - A v,
//             and partial sums of ||r||^2 and r^T r; computed in FP64.
//   OP_APPLY: v = x (input),  y = A v.
// The projector term uses ce[p] = e_kb[p] (v_p . v), prepared per CTA from the
// projections computed by the gather kernel; each grid point adds -sum over
// its atom entries of the projector values times ce.
#pragma once
#include <type_traits>

#include "cplx.cuh"
#include "ops_pair.cuh"
#include "rsn_internal.h"
#include "tma.cuh"

namespace rsn {

// FP32 operator value in difference form: the Laplacian is sum_m w_m sum over the
// six neighbours at distance m of (x_nb - x_c); near-equal values subtract
// exactly, so the large diagonal 3 c_0 / (2 h^2) never meets the small result
// for smooth fields.  dgv = (-V_loc, Gamma) without the FD diagonal.
template <typename C, typename CT, int R>
__device__ __forceinline__ C fd_diff_form(const C* qz, const C* smb, int so, int pitch, const CT* wst, C vc,
                                          float2 dgv, double E) {
  C lap = czero<C>();
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    C sm = cadd(csub(qz[R - m], vc), csub(qz[R + m], vc));
    sm = cadd(sm, cadd(csub(smb[so - m], vc), csub(smb[so + m], vc)));
    sm = cadd(sm, cadd(csub(smb[so - m * pitch], vc), csub(smb[so + m * pitch], vc)));
    lap = rfma(wst[m], sm, lap);
  }
  return cfma(mk2((CT)((float)E + dgv.x), (CT)dgv.y), vc, lap);
}

// Kahan-compensated accumulation (sum, carry) for long FP32 dot products.
template <typename S>
__device__ __forceinline__ void kahan_add(S& sum, S& carry, S term) {
  const S y = term - carry;
  const S t = sum + y;
  carry = (t - sum) - y;
  sum = t;
}

// y -= sum_j a_j cp[j] over one quad of an atom entry's projector values
// (FP64 values for an FP64 compute type, else FP32), in projector order.
template <typename C, typename CT>
__device__ __forceinline__ C proj_quad(const JuncDev& J, int qi, const C* cp, C y) {
  if constexpr (sizeof(CT) == 8) {
    const double2 a01 = J.inv_q64[2 * (size_t)qi], a23 = J.inv_q64[2 * (size_t)qi + 1];
    y = rfma((CT)-a01.x, cp[0], y);
    y = rfma((CT)-a01.y, cp[1], y);
    y = rfma((CT)-a23.x, cp[2], y);
    y = rfma((CT)-a23.y, cp[3], y);
  } else {
    const float4 a = J.inv_q32[qi];
    y = rfma((CT)-a.x, cp[0], y);
    y = rfma((CT)-a.y, cp[1], y);
    y = rfma((CT)-a.z, cp[2], y);
    y = rfma((CT)-a.w, cp[3], y);
  }
  return y;
}

template <typename T, int MODE> struct RawIn;
template <typename T> struct RawIn<T, OP_COCG> { typename cx<T>::t a, b; };
template <typename T> struct RawIn<T, OP_RESID> { double2 a; typename cx<T>::t b; };
template <typename T> struct RawIn<T, OP_APPLY> { typename cx<T>::t a; };

// At most kOpThreads threads per CTA; the minimum resident CTAs per SM bound
// the registers per thread (64 / 85 / 128 for 1 / 2 / 3+ points per thread,
// 128 for the FP64 true residual).
constexpr int kOpThreads = 256;

// One (tile, slot) of the operator: the CTA's tile blockIdx.x of slot s.
template <typename T, int R, int PPT, int MODE>
__device__ __forceinline__ void op_tile(const JuncDev* __restrict__ jt, const BatchDev& b, const int s,
                                        const void* __restrict__ x_in, void* __restrict__ y_out,
                                        const void* __restrict__ c_in) {
  // compute type: FP64 for the true residual, else the inner precision
  using CT = typename std::conditional<MODE == OP_RESID, double, T>::type;
  using C = typename cx<CT>::t;   // compute complex
  using CO = typename cx<T>::t;   // storage complex of the Krylov vectors
  using Raw = RawIn<T, MODE>;
  constexpr int Q = 2 * R + 1;
  constexpr int PF = 3;  // planes loaded ahead of use

  if constexpr (MODE == OP_COCG) {
    if (b.state[s] != SL_ACTIVE) return;
  } else if constexpr (MODE == OP_RESID) {
    const int stt = b.state[s];
    if (stt != SL_NEW && stt != SL_CHECK) return;
  }
  const JuncDev& J = jt[b.junc[s]];
  const int tile = blockIdx.x;
  if (tile >= J.nA || (MODE != OP_RESID && J.kind != kOpReg)) return;

  const int nx = J.nx, ny = J.ny, nz = J.nz, plane = J.plane, TY = J.TY;
  const int yt = tile % J.ytiles, zt = tile / J.ytiles;
  const int z0 = zt * J.Lz, z1 = min(z0 + J.Lz, nz);
  const int y0 = yt * TY, y1 = min(y0 + TY, ny), ty = y1 - y0;
  const int pitch = nx + 2 * R, rows = TY + 2 * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long vo = b.voff[s];
  const long long xo = (MODE == OP_RESID) ? b.xo[s] : 0;
  const double E = b.E[s];
  const double sig = (MODE == OP_RESID) ? b.sigma[s] : 1.0;  // d is stored in units of ||b||

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm0 = reinterpret_cast<C*>(smem_raw);
  C* sm1 = sm0 + rows * pitch;
  C* ce = sm1 + rows * pitch;
  __shared__ double red[32 * 4];

  for (int i = tid; i < 2 * rows * pitch; i += nt) sm0[i] = czero<C>();

  // ---- per-system scalars ---------------------------------------------------
  const int k = (MODE == OP_COCG) ? b.iters[s] : 0;
  const bool first = (MODE == OP_COCG) && (k == 0);
  C beta = czero<C>();
  if (MODE == OP_COCG && !first) beta = from64<C>(b.beta_cur[s]);
  const CO* pold = nullptr;
  CO* pnew = nullptr;
  if constexpr (MODE == OP_COCG) {
    pold = reinterpret_cast<const CO*>((k & 1) ? b.p1 : b.p0);
    pnew = reinterpret_cast<CO*>((k & 1) ? b.p0 : b.p1);
  }

  // ---- projector coefficients ce[p] = e_kb[p] * (v_p . v) -------------------
  // (COCG: none.  The projector term of q = A p is added by the update
  // kernel, and the projection kernel forms c_p = v_p . p of the new direction,
  // e_kb c_p and the term's share of mu, -sum_p e_kb[p] c_p^2 (p^T v_p = c_p,
  // unconjugated), from the projections alone.)
  const int n_proj = J.n_proj;
  if (MODE != OP_COCG && n_proj > 0) {
    if constexpr (MODE == OP_RESID) {
      const double2* cxp = b.c_x + (size_t)s * b.pstride;
      for (int p = tid; p < n_proj; p += nt) {
        const double e = J.ekb[p];
        ce[p] = mk2((CT)(e * cxp[p].x), (CT)(e * cxp[p].y));
      }
    } else {
      const CO* cin = reinterpret_cast<const CO*>(c_in) + (size_t)s * b.pstride;
      for (int p = tid; p < n_proj; p += nt) {
        const CT e = (CT)J.ekb[p];
        C c = cin[p];
        ce[p] = mk2(e * c.x, e * c.y);
      }
    }
    for (int p = tid; p < kCePad; p += nt) ce[n_proj + p] = czero<C>();
  }

  // ---- owned points and halo rows -----------------------------------------
  int po[PPT], so[PPT];
  bool own[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int t = tid + u * nt;
    own[u] = t < nx * ty;
    const int x = own[u] ? t % nx : 0, yl = own[u] ? t / nx : 0;
    po[u] = x + (y0 + yl) * nx;
    so[u] = (yl + R) * pitch + x + R;
  }
  const int hlo = min(R, y0), hhi = min(R, ny - y1);
  const int nhalo = nx * (hlo + hhi);

  // ---- raw loads and the producer -------------------------------------------
  const CO* rv = reinterpret_cast<const CO*>(b.r);
  auto load_raw = [&](long long gl) -> Raw {  // gl: index within the junction
    Raw w;
    if constexpr (MODE == OP_COCG) {
      w.a = rv[vo + gl];
      w.b = first ? czero<CO>() : pold[vo + gl];
    } else if constexpr (MODE == OP_RESID) {
      w.a = b.x64[xo + gl];
      w.b = reinterpret_cast<const CO*>(b.d)[vo + gl];
    } else {
      w.a = reinterpret_cast<const CO*>(x_in)[vo + gl];
    }
    return w;
  };
  auto zero_raw = [&]() -> Raw {
    Raw w;
    if constexpr (MODE == OP_COCG) { w.a = czero<CO>(); w.b = czero<CO>(); }
    else if constexpr (MODE == OP_RESID) { w.a = make_double2(0.0, 0.0); w.b = czero<CO>(); }
    else { w.a = czero<CO>(); }
    return w;
  };
  auto produce = [&](const Raw& w) -> C {
    if constexpr (MODE == OP_COCG) {
      C v = w.a;
      if (!first) v = cfma(beta, (C)w.b, v);
      return v;
    } else if constexpr (MODE == OP_RESID) {
      const double2 dd = to64(w.b);
      return mk2(fma(sig, dd.x, w.a.x), fma(sig, dd.y, w.a.y));
    } else {
      return (C)w.a;
    }
  };

  C qv[PPT][Q];
#pragma unroll
  for (int u = 0; u < PPT; ++u)
#pragma unroll
    for (int m = 0; m < Q; ++m) qv[u][m] = czero<C>();
  Raw pf[PF][PPT];
  // planes z0-R .. z0-R+PF-1 are in flight before the march starts
#pragma unroll
  for (int f = 0; f < PF; ++f) {
    const int zl = z0 - R + f;
#pragma unroll
    for (int u = 0; u < PPT; ++u)
      pf[f][u] = (own[u] && zl >= 0 && zl < nz) ? load_raw((long long)zl * plane + po[u]) : zero_raw();
  }

  CT wst[R + 1];
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    if constexpr (sizeof(CT) == 8) wst[m] = (CT)J.w64[m];
    else wst[m] = (CT)J.w32[m];
  }

  CT acc0 = 0, acc1 = 0, acc2 = 0;  // COCG: mu(re,im) ; RESID: nrm, rho(re,im)
  double acc3 = 0.0;                // RESID: sum Gamma_L |v|^2 of the iterate (T partial)
  CT car0 = 0, car1 = 0;            // Kahan carries of the COCG sums
  // per-point operator data of the next plane to compute, loaded one plane early
  float2 dgf_n[PPT];
  int e0_n[PPT], e1_n[PPT];
  auto load_pt = [&](int z) {
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      dgf_n[u] = make_float2(0.f, 0.f);
      e0_n[u] = e1_n[u] = 0;
      if (own[u] && z < z1) {
        const long long g = (long long)z * plane + po[u];
        if constexpr (sizeof(CT) == 4) dgf_n[u] = J.dg32[g];
        if (MODE != OP_COCG && n_proj > 0) {
          e0_n[u] = J.inv_ptr[g];
          e1_n[u] = J.inv_ptr[g + 1];
        }
      }
    }
  };
  load_pt(z0);
  __syncthreads();

  for (int zc = z0 - 2 * R; zc < z1; ++zc) {
    // plane zc + R enters the register queue; plane zc + R + PF is requested
    const int zn = zc + R + PF;
    const bool zin = (zn >= 0) && (zn < nz);
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
#pragma unroll
      for (int m = 0; m < Q - 1; ++m) qv[u][m] = qv[u][m + 1];
      qv[u][Q - 1] = produce(pf[0][u]);
#pragma unroll
      for (int f = 0; f < PF - 1; ++f) pf[f][u] = pf[f + 1][u];
      pf[PF - 1][u] = (own[u] && zin) ? load_raw((long long)zn * plane + po[u]) : zero_raw();
    }
    if (zc < z0) continue;

    C* smb = ((zc - z0) & 1) ? sm1 : sm0;
#pragma unroll
    for (int u = 0; u < PPT; ++u)
      if (own[u]) smb[so[u]] = qv[u][R];
    for (int hh = tid; hh < nhalo; hh += nt) {
      const int hr = hh / nx, x = hh - hr * nx;
      const int yl = (hr < hlo) ? (hr - hlo) : (ty + hr - hlo);
      smb[(yl + R) * pitch + x + R] = produce(load_raw((long long)zc * plane + (y0 + yl) * nx + x));
    }
    __syncthreads();
    float2 dgf_c[PPT];
    int e0_c[PPT], e1_c[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      dgf_c[u] = dgf_n[u];
      e0_c[u] = e0_n[u];
      e1_c[u] = e1_n[u];
    }
    load_pt(zc + 1);

#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      if (!own[u]) continue;
      const C vc = qv[u][R];
      const long long gl = (long long)zc * plane + po[u];  // index within the junction
      C y;
      if constexpr (sizeof(CT) == 8) {
        C lap = czero<C>();
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          C sm = cadd(qv[u][R - m], qv[u][R + m]);
          sm = cadd(sm, cadd(smb[so[u] - m], smb[so[u] + m]));
          sm = cadd(sm, cadd(smb[so[u] - m * pitch], smb[so[u] + m * pitch]));
          lap = rfma(wst[m], sm, lap);
        }
        const double2 t = J.dg64[gl];
        y = cfma(mk2((CT)(E + t.x), (CT)t.y), vc, lap);
      } else {
        y = fd_diff_form<C, CT, R>(qv[u], smb, so[u], pitch, wst, vc, dgf_c[u], E);
      }
      if (MODE != OP_COCG && n_proj > 0) {
        const int e0 = e0_c[u], e1 = e1_c[u], nq = J.inv_nq;
        for (int e = e0; e < e1; ++e) {
          const C* cp = ce + J.inv_p0[e];
          for (int qd = 0; qd < nq; ++qd) y = proj_quad<C, CT>(J, e * nq + qd, cp + 4 * qd, y);
        }
      }
      if constexpr (MODE == OP_COCG) {
        pnew[vo + gl] = vc;
        reinterpret_cast<CO*>(b.q)[vo + gl] = y;
        kahan_add(acc0, car0, fma(vc.x, y.x, -vc.y * y.y));
        kahan_add(acc1, car1, fma(vc.x, y.y, vc.y * y.x));
      } else if constexpr (MODE == OP_RESID) {
        double2 bb = make_double2(0.0, 0.0);
        const int col = b.col[s];
        if (col >= 0) {
          if (gl == col) bb.x = 1.0;
        } else {
          const double g = J.gl[gl];
          if (g > 0.0) {
            const double2 xf = b.xf[b.xfo[s] + gl];
            bb = make_double2(g * xf.x, -g * xf.y);
          }
        }
        const CO rt = from64<CO>(make_double2(bb.x - (double)y.x, bb.y - (double)y.y));
        reinterpret_cast<CO*>(b.r)[vo + gl] = rt;
        const double rx = rt.x, ry = rt.y;
        acc0 = fma(rx, rx, fma(ry, ry, acc0));
        acc1 = fma(rx, rx, fma(-ry, ry, acc1));
        acc2 = fma(2.0 * rx, ry, acc2);
        if (col >= 0) {
          const double g = J.gl[gl];
          acc3 = fma(g, (double)vc.x * vc.x + (double)vc.y * vc.y, acc3);
        }
      } else {
        reinterpret_cast<CO*>(y_out)[vo + gl] = from64<CO>(to64(y));
      }
    }
  }

  if constexpr (MODE == OP_COCG) {
    CT v[2] = {acc0 - car0, acc1 - car1};
    double out[2];
    block_sum<2>(v, red, out);
    if (tid == 0) b.mu_part[(size_t)s * b.PA + tile] = make_double2(out[0], out[1]);
  } else if constexpr (MODE == OP_RESID) {
    CT v[4] = {acc0, acc1, acc2, acc3};
    double out[4];
    block_sum<4>(v, red, out);
    if (tid == 0) {
      b.t0_part[(size_t)s * b.PA + tile] = out[3];
      b.nrm0_part[(size_t)s * b.PA + tile] = out[0];
      b.rho0_part[(size_t)s * b.PA + tile] = make_double2(out[1], out[2]);
    }
  }
}

template <typename T, int R, int PPT, int MODE>
__global__ void __launch_bounds__(kOpThreads, (MODE == OP_RESID ? 2 : (PPT == 1 ? 4 : (PPT == 2 ? 3 : 2))))
op_kernel(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp, const void* __restrict__ x_in,
          void* __restrict__ y_out, const void* __restrict__ c_in) {
  const BatchDev& b = *bp;
  if constexpr (MODE == OP_RESID) {
    // the true residual runs only for the NEW / CHECK slots of the list: CTA
    // rows take its entries in turn
    const int n = *b.lst_n;
    for (int li = blockIdx.y; li < n; li += gridDim.y) {
      op_tile<T, R, PPT, MODE>(jt, b, b.lst[li], x_in, y_out, c_in);
      __syncthreads();  // the shared-memory planes are reused by the next entry
    }
  } else {
    op_tile<T, R, PPT, MODE>(jt, b, blockIdx.y, x_in, y_out, c_in);
  }
}

template <int R>
cudaError_t launch_op_r(int mode, bool fp32, int ppt, dim3 grid, int threads, size_t smem, cudaStream_t st,
                        const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  void (*kern)(const JuncDev*, const BatchDev*, const void*, void*, const void*) = nullptr;
#define RSN_PICK(T, P)                                                   \
  if (mode == OP_COCG) kern = op_kernel<T, R, P, OP_COCG>;               \
  else if (mode == OP_RESID) kern = op_kernel<T, R, P, OP_RESID>;        \
  else kern = op_kernel<T, R, P, OP_APPLY>;
  if (fp32) {
    switch (ppt) {
      case 1: RSN_PICK(float, 1) break;
      case 2: RSN_PICK(float, 2) break;
      case 3: RSN_PICK(float, 3) break;
      case 4: RSN_PICK(float, 4) break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (ppt) {
      case 1: RSN_PICK(double, 1) break;
      case 2: RSN_PICK(double, 2) break;
      case 3: RSN_PICK(double, 3) break;
      case 4: RSN_PICK(double, 4) break;
      default: return cudaErrorInvalidValue;
    }
  }
#undef RSN_PICK
  if (smem > 48 * 1024) {
    cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  kern<<<grid, threads, smem, st>>>(jt, b, x_in, y_out, c_in);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Plane-streaming variant for tiles that are whole x-y planes (TY = ny, at most
// 1024 points): the inputs of each plane (r and p_old, or x) arrive by bulk
// copies (TMA) in a ring of kStages shared-memory stages, issued kStages
// planes ahead, so the bytes in flight do not occupy registers.  One thread
// per grid point keeps only the 2R+1-deep z queue.  Used for OP_COCG and
// OP_APPLY when every plane and slot offset is 16-byte aligned.
// ---------------------------------------------------------------------------
constexpr int kStages = 4;

template <typename T, int R, int MODE>
__global__ void __launch_bounds__(1024, 1)
op_kernel_tma(const JuncDev* __restrict__ jt, const BatchDev* __restrict__ bp, const void* __restrict__ x_in,
              void* __restrict__ y_out, const void* __restrict__ c_in) {
  using C = typename cx<T>::t;
  constexpr int Q = 2 * R + 1;
  constexpr int NIN = (MODE == OP_COCG) ? 2 : 1;
  const BatchDev& b = *bp;
  const int s = blockIdx.y;
  if constexpr (MODE == OP_COCG) {
    if (b.state[s] != SL_ACTIVE) return;
  }
  const JuncDev& J = jt[b.junc[s]];
  const int tile = blockIdx.x;
  if (tile >= J.nA || J.kind != kOpTma) return;
  const int nx = J.nx, ny = J.ny, nz = J.nz, plane = J.plane;
  const int z0 = tile * J.Lz, z1 = min(z0 + J.Lz, nz);
  const int pitch = nx + 2 * R, prow = ny + 2 * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long vo = b.voff[s];
  const double E = b.E[s];

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* stage = reinterpret_cast<C*>(smem_raw);          // [kStages][NIN][plane]
  C* exch = stage + kStages * NIN * plane;           // [2][prow][pitch]
  C* ce = exch + 2 * prow * pitch;                   // [n_proj]
  const int n_proj = J.n_proj;
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(ce + n_proj + kCePad) + 15) & ~static_cast<uintptr_t>(15));
  __shared__ double red[32 * 2];
  __shared__ int s_bad;

  for (int i = tid; i < 2 * prow * pitch; i += nt) exch[i] = czero<C>();
  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(bars + k, 1);
    s_bad = 0;
  }

  const int k = (MODE == OP_COCG) ? b.iters[s] : 0;
  const bool first = (MODE == OP_COCG) && (k == 0);
  C beta = czero<C>();
  if (MODE == OP_COCG && !first) beta = from64<C>(b.beta_cur[s]);
  const C* src0;
  const C* src1 = nullptr;
  C* pnew = nullptr;
  if constexpr (MODE == OP_COCG) {
    src0 = reinterpret_cast<const C*>(b.r) + vo;
    if (!first) src1 = reinterpret_cast<const C*>((k & 1) ? b.p1 : b.p0) + vo;
    pnew = reinterpret_cast<C*>((k & 1) ? b.p0 : b.p1);
  } else {
    src0 = reinterpret_cast<const C*>(x_in) + vo;
  }
  // APPLY only: in COCG the projector term of q is added on the support points
  if (MODE != OP_COCG && n_proj > 0) {
    const C* cin = reinterpret_cast<const C*>(c_in) + (size_t)s * b.pstride;
    for (int p = tid; p < n_proj; p += nt) {
      const T e = (T)J.ekb[p];
      const C c = cin[p];
      ce[p] = mk2(e * c.x, e * c.y);
    }
    for (int p = tid; p < kCePad; p += nt) ce[n_proj + p] = czero<C>();
  }
  __syncthreads();

  // planes [zb, ze) stream through the ring; plane zl uses stage (zl - zb) % kStages
  const int zb = z0 - R, ze = z1 + R;
  const uint32_t pbytes = (uint32_t)(plane * sizeof(C));
  auto issue = [&](int zl) {
    const int st = (zl - zb) % kStages;
    uint64_t* bar = bars + st;
    if (zl >= 0 && zl < nz) {
      mbar_arrive_expect_tx(bar, src1 ? 2 * pbytes : pbytes);
      bulk_g2s(stage + (st * NIN) * plane, src0 + (size_t)zl * plane, pbytes, bar);
      if (src1) bulk_g2s(stage + (st * NIN + 1) * plane, src1 + (size_t)zl * plane, pbytes, bar);
    } else {
      mbar_arrive(bar);  // nothing to copy outside the box: complete the phase
    }
  };
  if (tid == 0)
    for (int f = 0; f < kStages && zb + f < ze; ++f) issue(zb + f);

  const bool own = tid < plane;
  const int xx = own ? tid % nx : 0, yy = own ? tid / nx : 0;
  const int so = (yy + R) * pitch + xx + R;
  T wst[R + 1];
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    if constexpr (sizeof(T) == 8) wst[m] = (T)J.w64[m];
    else wst[m] = (T)J.w32[m];
  }
  C qv[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) qv[m] = czero<C>();
  T acc0 = 0, acc1 = 0, car0 = 0, car1 = 0;
  // per-point operator data of the next plane to compute, loaded one plane early
  float2 dg_n = make_float2(0.f, 0.f);
  int e0_n = 0, e1_n = 0;
  auto load_pt = [&](int z) {
    if (own && z < z1) {
      const long long g = (long long)z * plane + tid;
      if constexpr (sizeof(T) == 4) dg_n = J.dg32[g];
      if (MODE != OP_COCG && n_proj > 0) {
        e0_n = J.inv_ptr[g];
        e1_n = J.inv_ptr[g + 1];
      }
    }
  };
  load_pt(z0);

  for (int zc = z0 - 2 * R; zc < z1; ++zc) {
    const int zl = zc + R;
    const int st = (zl - zb) % kStages;
    C v = czero<C>();
    if (!mbar_wait(bars + st, (uint32_t)(((zl - zb) / kStages) & 1))) {
      s_bad = 1;
    } else if (own && zl >= 0 && zl < nz) {
      v = stage[(st * NIN) * plane + tid];
      if (src1) v = cfma(beta, stage[(st * NIN + 1) * plane + tid], v);
    }
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) qv[m] = qv[m + 1];
    qv[Q - 1] = v;
    C* smb = exch + (((zc - z0) & 1) ? prow * pitch : 0);
    if (zc >= z0 && own) smb[so] = qv[R];
    __syncthreads();
    if (s_bad) {
      // a copy never arrived: report, let in-flight copies land (bounded), leave
      if (tid == 0) {
        if (b.sched) atomicExch(b.sched + 2, 1);
        for (int f = 0; f < kStages; ++f) {
          const int zq = zl + f;
          if (zq < ze) mbar_wait(bars + (zq - zb) % kStages, (uint32_t)(((zq - zb) / kStages) & 1));
        }
      }
      return;
    }
    if (tid == 0 && zl + kStages < ze) {
      fence_proxy_async();
      issue(zl + kStages);
    }
    if (zc < z0 || !own) continue;
    const float2 dg_c = dg_n;
    const int e0 = e0_n, e1 = e1_n;
    load_pt(zc + 1);

    const C vc = qv[R];
    const long long gl = (long long)zc * plane + tid;
    C y;
    if constexpr (sizeof(T) == 8) {
      C lap = czero<C>();
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        C sm = cadd(qv[R - m], qv[R + m]);
        sm = cadd(sm, cadd(smb[so - m], smb[so + m]));
        sm = cadd(sm, cadd(smb[so - m * pitch], smb[so + m * pitch]));
        lap = rfma(wst[m], sm, lap);
      }
      const double2 t = J.dg64[gl];
      y = cfma(mk2((T)(E + t.x), (T)t.y), vc, lap);
    } else {
      y = fd_diff_form<C, T, R>(qv, smb, so, pitch, wst, vc, dg_c, E);
    }
    if (MODE != OP_COCG && n_proj > 0) {
      const int nq = J.inv_nq;
      for (int e = e0; e < e1; ++e) {
        const C* cp = ce + J.inv_p0[e];
        for (int qd = 0; qd < nq; ++qd) y = proj_quad<C, T>(J, e * nq + qd, cp + 4 * qd, y);
      }
    }
    if constexpr (MODE == OP_COCG) {
      pnew[vo + gl] = vc;
      reinterpret_cast<C*>(b.q)[vo + gl] = y;
      kahan_add(acc0, car0, fma(vc.x, y.x, -vc.y * y.y));
      kahan_add(acc1, car1, fma(vc.x, y.y, vc.y * y.x));
    } else {
      reinterpret_cast<C*>(y_out)[vo + gl] = y;
    }
  }
  if constexpr (MODE == OP_COCG) {
    T vv[2] = {acc0 - car0, acc1 - car1};
    double out[2];
    block_sum<2>(vv, red, out);
    if (tid == 0) b.mu_part[(size_t)s * b.PA + tile] = make_double2(out[0], out[1]);
  }
}

template <int R>
cudaError_t launch_op_tma_r(int mode, bool fp32, dim3 grid, int threads, size_t smem, cudaStream_t st,
                            const JuncDev* jt, const BatchDev* b, const void* x_in, void* y_out, const void* c_in) {
  void (*kern)(const JuncDev*, const BatchDev*, const void*, void*, const void*) = nullptr;
  if (mode == OP_COCG) kern = fp32 ? op_kernel_tma<float, R, OP_COCG> : op_kernel_tma<double, R, OP_COCG>;
  else if (mode == OP_APPLY) kern = fp32 ? op_kernel_tma<float, R, OP_APPLY> : op_kernel_tma<double, R, OP_APPLY>;
  else return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  kern<<<grid, threads, smem, st>>>(jt, b, x_in, y_out, c_in);
  return cudaGetLastError();
}

}  // namespace rsn

#define RSN_INSTANTIATE_OPS(R)                                                                    \
  namespace rsn {                                                                                 \
  cudaError_t launch_op_R##R(int mode, bool fp32, int ppt, dim3 grid, int threads, size_t smem,  \
                             cudaStream_t st, const JuncDev* jt, const BatchDev* b,             \
                             const void* x_in, void* y_out, const void* c_in) {                  \
    return launch_op_r<R>(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);   \
  }                                                                                               \
  cudaError_t launch_op_tma_R##R(int mode, bool fp32, dim3 grid, int threads, size_t smem,        \
                                 cudaStream_t st, const JuncDev* jt, const BatchDev* b,         \
                                 const void* x_in, void* y_out, const void* c_in) {              \
    return launch_op_tma_r<R>(mode, fp32, grid, threads, smem, st, jt, b, x_in, y_out, c_in);    \
  }                                                                                               \
  cudaError_t launch_op_plane_R##R(int mode, dim3 grid, int threads, size_t smem, cudaStream_t st, \
                                   const JuncDev* jt, const BatchDev* b, const void* x_in,      \
                                   void* y_out, const void* c_in) {                              \
    return launch_op_plane_r<R>(mode, grid, threads, smem, st, jt, b, x_in, y_out, c_in);        \
  }                                                                                               \
  cudaError_t launch_op_pair_R##R(int mode, bool big, dim3 grid, int threads, size_t smem,        \
                                  cudaStream_t st, const JuncDev* jt, const BatchDev* b,        \
                                  const void* x_in, void* y_out, const void* c_in) {             \
    return launch_op_pair_r<R>(mode, big, grid, threads, smem, st, jt, b, x_in, y_out, c_in);    \
  }                                                                                               \
  }
