// Small complex helpers on float2 / double2 (interleaved re, im) and the
// deterministic block reductions used by every kernel.
#pragma once
#include <cuda_runtime.h>

namespace rsn {

template <typename T> struct cx;
template <> struct cx<float> { using t = float2; };
template <> struct cx<double> { using t = double2; };

__host__ __device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// a * b (complex)
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// acc + a * b (complex)
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}
// acc + s * a (s real)
template <typename C, typename S> __device__ __forceinline__ C rfma(S s, C a, C acc) {
  acc.x = fma(s, a.x, acc.x); acc.y = fma(s, a.y, acc.y); return acc;
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double2 to64(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to64(double2 a) { return a; }
template <typename C> __device__ __forceinline__ C from64(double2 a);
template <> __device__ __forceinline__ float2 from64<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 from64<double2>(double2 a) { return a; }

// Sum NV values over the CTA in a fixed order (warp shuffle tree, then warps in
// index order).  Warp stages run in the accumulator type; the cross-warp stage
// in double.  Result valid in thread 0.  `red` must hold 32*NV doubles.
template <int NV, typename A>
__device__ __forceinline__ void block_sum(A (&v)[NV], double* red, double (&out)[NV]) {
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) red[warp * NV + i] = (double)v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w * NV + i];
      out[i] = s;
    }
  }
  __syncthreads();
}

// Allow `smem` bytes of dynamic shared memory for kernel `kern`: the attribute
// is set to the device's opt-in maximum less the kernel's static shared memory
// (not to this launch's size: contexts on other host threads may launch the
// same kernel with other sizes concurrently).
inline cudaError_t set_max_dynamic_smem(const void* kern, size_t smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  const long long room = (long long)optin - (long long)fa.sharedSizeBytes;
  if (room < (long long)smem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
}

}  // namespace rsn
