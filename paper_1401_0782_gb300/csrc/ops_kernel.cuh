// Operator kernel: y = A(E) v with A(E) = E - H_KS + i(Gamma_L + Gamma_R)
// (Eqs. G and Hop), H_KS = -1/2 lap_FD + V_loc + sum_p |v_p> e_kb <v_p| (Sec. II.C).
//
// One CTA owns a tile of full x rows (y rows [y0, y0+TY)) and z planes
// [z0, z0+Lz) of one system s, and marches along z.  Each thread owns PPT
// (x, y) columns of the tile and keeps the 2R+1 planes around the current one
// in registers, so z neighbours are never re-read.  The current plane (plus R
// halo rows above and below, zero outside the box) is exchanged through a
// double-buffered shared-memory tile for the x and y neighbours: one barrier
// per plane.  Every vector element is read from memory once per tile (plus
// 2R halo planes per z chunk and the halo rows of y tiles).
//
// The value fed to the stencil is produced on the fly, which fuses the
// neighbouring vector update into the matvec:
//   OP_COCG : v = r + beta p_old   (COCG direction update), writes p_new = v,
//             q = A v and the partial sums of mu = v^T q (unconjugated).
//   OP_RESID: v = x64 + d          (refinement iterate), writes r = b - A v,
//             and partial sums of ||r||^2 and r^T r; computed in FP64.
//   OP_APPLY: v = x (input),  y = A v.
// The projector term uses ce[p] = e_kb[p] (v_p . v), prepared per CTA from the
// projections computed by the gather kernel; each grid point adds
// -sum over its (p, value) entries.
#pragma once
#include <type_traits>

#include "cplx.cuh"
#include "rsn_internal.h"

namespace rsn {

// rho_k of slot s: k = 0 comes from the true-residual kernel, k >= 1 from the
// COCG update kernel (double-buffered by iteration parity).  Fixed-order sums.
__device__ __forceinline__ double2 slot_rho(const BatchDev& b, const JuncDev& J, int s, int k) {
  double2 acc = make_double2(0.0, 0.0);
  if (k == 0) {
    const double2* p = b.rho0_part + (size_t)s * b.PA;
    for (int t = 0; t < J.nR; ++t) { acc.x += p[t].x; acc.y += p[t].y; }
  } else {
    const double2* p = b.rho_part + ((size_t)(k & 1) * b.nslots + s) * b.PB;
    for (int t = 0; t < J.nB; ++t) { acc.x += p[t].x; acc.y += p[t].y; }
  }
  return acc;
}

template <typename T, int R, int PPT, int MODE>
__global__ void __launch_bounds__(512)
op_kernel(const JuncDev* __restrict__ jt, const BatchDev b, const void* __restrict__ x_in,
          void* __restrict__ y_out, const void* __restrict__ c_in) {
  // compute type: FP64 for the true residual, else the inner precision
  using CT = typename std::conditional<MODE == OP_RESID, double, T>::type;
  using C = typename cx<CT>::t;   // compute complex
  using CO = typename cx<T>::t;   // storage complex of the Krylov vectors
  constexpr int Q = 2 * R + 1;

  const int s = blockIdx.y;
  if (MODE == OP_COCG && b.done[s]) return;
  if (MODE == OP_RESID && b.outer_done[s]) return;
  const JuncDev& J = jt[b.junc[s]];
  const int tile = blockIdx.x;
  if (tile >= J.nA) return;

  const int nx = J.nx, ny = J.ny, nz = J.nz, plane = J.plane, TY = J.TY;
  const int yt = tile % J.ytiles, zt = tile / J.ytiles;
  const int z0 = zt * J.Lz, z1 = min(z0 + J.Lz, nz);
  const int y0 = yt * TY, y1 = min(y0 + TY, ny), ty = y1 - y0;
  const int pitch = nx + 2 * R, rows = TY + 2 * R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long vo = b.voff[s];
  const double E = b.E[s];

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm0 = reinterpret_cast<C*>(smem_raw);
  C* sm1 = sm0 + rows * pitch;
  C* ce = sm1 + rows * pitch;
  __shared__ double red[32 * 3];

  for (int i = tid; i < 2 * rows * pitch; i += nt) sm0[i] = czero<C>();

  // ---- per-system scalars ---------------------------------------------------
  const int k = (MODE == OP_COCG) ? b.iters[s] : 0;
  const bool first = (MODE == OP_COCG) && (k == 0);
  C beta = czero<C>();
  if (MODE == OP_COCG && !first) {
    double2 bt = cdiv(slot_rho(b, J, s, k), slot_rho(b, J, s, k - 1));
    beta = from64<C>(bt);
  }
  const CO* pold = nullptr;
  CO* pnew = nullptr;
  if constexpr (MODE == OP_COCG) {
    pold = reinterpret_cast<const CO*>((k & 1) ? b.p1 : b.p0);
    pnew = reinterpret_cast<CO*>((k & 1) ? b.p0 : b.p1);
  }

  // ---- projector coefficients ce[p] = e_kb[p] * (v_p . v) -------------------
  const int n_proj = J.n_proj;
  if (n_proj > 0) {
    if constexpr (MODE == OP_COCG) {
      const CO* cr = reinterpret_cast<const CO*>(b.c_r) + (size_t)s * n_proj;
      const CO* cpo = reinterpret_cast<const CO*>(b.c_p) + ((size_t)(k & 1) * b.nslots + s) * n_proj;
      CO* cpn = reinterpret_cast<CO*>(b.c_p) + ((size_t)((k + 1) & 1) * b.nslots + s) * n_proj;
      for (int p = tid; p < n_proj; p += nt) {
        C c = cr[p];
        if (!first) c = cfma(beta, (C)cpo[p], c);
        if (tile == 0) cpn[p] = c;
        const CT e = (CT)J.ekb[p];
        ce[p] = mk2(e * c.x, e * c.y);
      }
    } else if constexpr (MODE == OP_RESID) {
      const double2* cxp = b.c_x + (size_t)s * n_proj;
      for (int p = tid; p < n_proj; p += nt) {
        const double e = J.ekb[p];
        ce[p] = mk2((CT)(e * cxp[p].x), (CT)(e * cxp[p].y));
      }
    } else {
      const CO* cin = reinterpret_cast<const CO*>(c_in) + (size_t)s * n_proj;
      for (int p = tid; p < n_proj; p += nt) {
        const CT e = (CT)J.ekb[p];
        C c = cin[p];
        ce[p] = mk2(e * c.x, e * c.y);
      }
    }
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

  // ---- producer: the vector the stencil acts on ----------------------------
  const CO* rv = reinterpret_cast<const CO*>(b.r);
  auto produce = [&](long long gi) -> C {
    if constexpr (MODE == OP_COCG) {
      C v = rv[gi];
      if (!first) v = cfma(beta, (C)pold[gi], v);
      return v;
    } else if constexpr (MODE == OP_RESID) {
      const double2 xx = b.x64[gi];
      const double2 dd = to64(reinterpret_cast<const CO*>(b.d)[gi]);
      return mk2(xx.x + dd.x, xx.y + dd.y);
    } else {
      return (C)(reinterpret_cast<const CO*>(x_in)[gi]);
    }
  };

  C qv[PPT][Q];
#pragma unroll
  for (int u = 0; u < PPT; ++u)
#pragma unroll
    for (int m = 0; m < Q; ++m) qv[u][m] = czero<C>();

  CT wst[R + 1];
#pragma unroll
  for (int m = 1; m <= R; ++m) wst[m] = (sizeof(CT) == 8) ? (CT)J.w64[m] : (CT)J.w32[m];

  CT acc0 = 0, acc1 = 0, acc2 = 0;  // COCG: mu(re,im) ; RESID: nrm, rho(re,im)
  __syncthreads();

  for (int zc = z0 - 2 * R; zc < z1; ++zc) {
    const int zl = zc + R;
    const bool zin = (zl >= 0) && (zl < nz);
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
#pragma unroll
      for (int m = 0; m < Q - 1; ++m) qv[u][m] = qv[u][m + 1];
      qv[u][Q - 1] = (own[u] && zin) ? produce(vo + (long long)zl * plane + po[u]) : czero<C>();
    }
    if (zc < z0) continue;

    C* smb = ((zc - z0) & 1) ? sm1 : sm0;
#pragma unroll
    for (int u = 0; u < PPT; ++u)
      if (own[u]) smb[so[u]] = qv[u][R];
    for (int hh = tid; hh < nhalo; hh += nt) {
      const int hr = hh / nx, x = hh - hr * nx;
      const int yl = (hr < hlo) ? (hr - hlo) : (ty + hr - hlo);
      smb[(yl + R) * pitch + x + R] = produce(vo + (long long)zc * plane + (y0 + yl) * nx + x);
    }
    __syncthreads();

#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      if (!own[u]) continue;
      const C vc = qv[u][R];
      C lap = czero<C>();
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        C sm = cadd(qv[u][R - m], qv[u][R + m]);
        sm = cadd(sm, cadd(smb[so[u] - m], smb[so[u] + m]));
        sm = cadd(sm, cadd(smb[so[u] - m * pitch], smb[so[u] + m * pitch]));
        lap = rfma(wst[m], sm, lap);
      }
      const long long gl = (long long)zc * plane + po[u];  // index within the junction
      C dg;
      if constexpr (sizeof(CT) == 8) {
        const double2 t = J.dg64[gl];
        dg = mk2((CT)(E + t.x), (CT)t.y);
      } else {
        const float2 t = J.dg32[gl];
        dg = mk2((CT)((float)E + t.x), (CT)t.y);
      }
      C y = cfma(dg, vc, lap);
      if (n_proj > 0) {
        const int e0 = J.inv_ptr[gl], e1 = J.inv_ptr[gl + 1];
        for (int e = e0; e < e1; ++e) {
          const CT a = (sizeof(CT) == 8) ? (CT)J.inv_val64[e] : (CT)J.inv_val32[e];
          y = rfma(-a, ce[J.inv_proj[e]], y);
        }
      }
      const long long gi = vo + gl;
      if constexpr (MODE == OP_COCG) {
        pnew[gi] = vc;
        reinterpret_cast<CO*>(b.q)[gi] = y;
        acc0 = fma(vc.x, y.x, fma(-vc.y, y.y, acc0));
        acc1 = fma(vc.x, y.y, fma(vc.y, y.x, acc1));
      } else if constexpr (MODE == OP_RESID) {
        double2 bb = make_double2(0.0, 0.0);
        const int col = b.col[s];
        if (col >= 0) {
          if (gl == col) bb.x = 1.0;
        } else {
          const double g = J.gl[gl];
          if (g > 0.0) {
            const double2 xf = b.xf[gi];
            bb = make_double2(g * xf.x, -g * xf.y);
          }
        }
        const CO rt = from64<CO>(make_double2(bb.x - (double)y.x, bb.y - (double)y.y));
        reinterpret_cast<CO*>(b.r)[gi] = rt;
        const double rx = rt.x, ry = rt.y;
        acc0 = fma(rx, rx, fma(ry, ry, acc0));
        acc1 = fma(rx, rx, fma(-ry, ry, acc1));
        acc2 = fma(2.0 * rx, ry, acc2);
      } else {
        reinterpret_cast<CO*>(y_out)[gi] = from64<CO>(to64(y));
      }
    }
  }

  if constexpr (MODE == OP_COCG) {
    CT v[2] = {acc0, acc1};
    double out[2];
    block_sum<2>(v, red, out);
    if (tid == 0) b.mu_part[(size_t)s * b.PA + tile] = make_double2(out[0], out[1]);
  } else if constexpr (MODE == OP_RESID) {
    CT v[3] = {acc0, acc1, acc2};
    double out[3];
    block_sum<3>(v, red, out);
    if (tid == 0) {
      b.nrm0_part[(size_t)s * b.PA + tile] = out[0];
      b.rho0_part[(size_t)s * b.PA + tile] = make_double2(out[1], out[2]);
    }
  }
}

template <int R>
cudaError_t launch_op_r(int mode, bool fp32, int ppt, dim3 grid, int threads, size_t smem,
                        cudaStream_t st, const JuncDev* jt, const BatchDev& b, const void* x_in,
                        void* y_out, const void* c_in) {
  void (*kern)(const JuncDev*, const BatchDev, const void*, void*, const void*) = nullptr;
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
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, threads, smem, st>>>(jt, b, x_in, y_out, c_in);
  return cudaGetLastError();
}

}  // namespace rsn

#define RSN_INSTANTIATE_OPS(R)                                                                    \
  namespace rsn {                                                                                 \
  cudaError_t launch_op_R##R(int mode, bool fp32, int ppt, dim3 grid, int threads, size_t smem,  \
                             cudaStream_t st, const JuncDev* jt, const BatchDev& b,             \
                             const void* x_in, void* y_out, const void* c_in) {                  \
    return launch_op_r<R>(mode, fp32, ppt, grid, threads, smem, st, jt, b, x_in, y_out, c_in);   \
  }                                                                                               \
  }
