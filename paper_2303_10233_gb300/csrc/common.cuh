// Shared definitions of the GB300 Q2--Q1* solver library (device + host).
//
// Quadrature: every element integral uses the 3x3 Gauss-Legendre rule on the
// affine map of a rectangle; on the reference interval [0,1] the points are
// 1/2 - sqrt(3/5)/2, 1/2, 1/2 + sqrt(3/5)/2 with weights 5/18, 8/18, 5/18.
// Shape functions on [0,1]: quadratic Lagrange at {0, 1/2, 1} for velocity,
// linear Lagrange at {0, 1} for the Q1 pressure, indicator for P0.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include "eth.h"

// Every kernel starts by waiting for the grids it depends on (griddepcontrol.wait).
// Outside a programmatic dependency this returns at once; inside the captured
// solver graphs the kernel-to-kernel edges are programmatic (the downstream
// grid is launched once all blocks of the upstream grid have started), so the
// wait is what orders a kernel after its producer and makes its writes visible.
#define ETH_GRID_DEP_WAIT() asm volatile("griddepcontrol.wait;\n" ::: "memory")

namespace eth {

constexpr double GOFF = 0.38729833462074168852;   // sqrt(3/5)/2
__host__ __device__ constexpr double gq(int q) { return q == 0 ? 0.5 - GOFF : (q == 1 ? 0.5 : 0.5 + GOFF); }
__host__ __device__ constexpr double gw(int q) { return q == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }
// quadratic Lagrange basis on [0,1] and its derivative
__host__ __device__ constexpr double q2v(int a, double t) {
  return a == 0 ? 2.0 * (t - 0.5) * (t - 1.0) : (a == 1 ? -4.0 * t * (t - 1.0) : 2.0 * t * (t - 0.5));
}
__host__ __device__ constexpr double q2d(int a, double t) {
  return a == 0 ? 4.0 * t - 3.0 : (a == 1 ? 4.0 - 8.0 * t : 4.0 * t - 1.0);
}
// linear Lagrange basis on [0,1]
__host__ __device__ constexpr double q1v(int c, double t) { return c == 0 ? 1.0 - t : t; }
__host__ __device__ constexpr double q1d(int c) { return c == 0 ? -1.0 : 1.0; }

// Table values at Gauss point q (compile-time when q, a are constants).
#define LV(q, a) ((CT)::eth::q2v((a), ::eth::gq(q)))
#define LD(q, a) ((CT)::eth::q2d((a), ::eth::gq(q)))
#define NV(q, c) ((CT)::eth::q1v((c), ::eth::gq(q)))
#define GW(q) ((CT)::eth::gw(q))

// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversions by integer operations on the IEEE-754 bit fields.
// On GB300 the hardware conversion instruction runs at the (reduced) FP64
// rate, which makes it the bottleneck of an FP32 element kernel with FP64
// inputs and outputs; the integer ALUs are not limited that way.
// binary64 -> binary32: rebias the exponent (1023 -> 127), keep the top 23
// mantissa bits and round half up on the first discarded bit (error <= 1/2
// ulp; the carry propagates into the exponent, overflowing to infinity).
// Magnitudes below the smallest normal binary32 become signed zero.
// binary32 -> binary64 is exact for normal numbers (subnormals become zero).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sign = hi & 0x80000000u;
  const unsigned e64 = (hi >> 20) & 0x7ffu;
  const int e = (int)e64 - 896;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned bits;
  if (e64 == 0x7ffu) bits = sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
  else if (e <= 0) bits = sign;
  else if (e >= 255) bits = sign | 0x7f800000u;
  else bits = (sign | ((unsigned)e << 23) | m) + ((lo >> 28) & 1u);
  return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned m = b & 0x7fffffu;
  unsigned hi, lo;
  if (e == 0u) { hi = sign; lo = 0u; }
  else if (e == 255u) { hi = sign | 0x7ff00000u | (m >> 3); lo = m << 29; }
  else { hi = sign | ((e + 896u) << 20) | (m >> 3); lo = m << 29; }
  return __hiloint2double((int)hi, (int)lo);
}

// The same rounding with a shorter common path.  Adding 2^28 to the 64-bit
// pattern rounds half up at the first dropped bit (the carry runs into the
// exponent); bits 60..29 then hold the low nine exponent bits and the 23 kept
// mantissa bits, and adding 128 to that nine-bit exponent field (mod 2^9) is
// the rebias 1023 -> 127 for every exponent of the normal binary32 range.
// Values outside that range (zero, binary32 subnormals, overflow, inf, NaN)
// take the full conversion above on the lanes that need it.
__device__ __forceinline__ float f64_to_f32_fast(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32);
  const unsigned t = (unsigned)((u + (1ull << 28)) >> 29) + 0x40000000u;
  const unsigned bits = (t & 0x7fffffffu) | (hi & 0x80000000u);
  const unsigned ea = hi & 0x7ff00000u;
  if (ea - (897u << 20) >= (254u << 20)) return f64_to_f32_bits(x);
  return __uint_as_float(bits);
}

// Warp-collective form for staged loads: lanes with valid == false yield 0
// without a conversion, and the full conversion runs only when some lane of
// the warp holds a value outside the normal binary32 range.  Every lane of
// the warp must call it (full mask).
__device__ __forceinline__ float f64_to_f32_warp(double x, bool valid) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32);
  const unsigned t = (unsigned)((u + (1ull << 28)) >> 29) + 0x40000000u;
  const unsigned bits = (t & 0x7fffffffu) | (hi & 0x80000000u);
  const bool out = valid && ((hi & 0x7ff00000u) - (897u << 20) >= (254u << 20));
  float r = valid ? __uint_as_float(bits) : 0.0f;
  if (__any_sync(0xffffffffu, out)) {
    if (out) r = f64_to_f32_bits(x);
  }
  return r;
}

#ifndef ETH_IN_FASTCVT
#define ETH_IN_FASTCVT 1
#endif

template <class TO, class TI>
__device__ __forceinline__ TO cvt(TI v) { return (TO)v; }
template <>
__device__ __forceinline__ float cvt<float, double>(double v) {
#if ETH_IN_FASTCVT
  return f64_to_f32_fast(v);
#else
  return f64_to_f32_bits(v);
#endif
}
template <>
__device__ __forceinline__ double cvt<double, float>(float v) { return f32_to_f64_bits(v); }

// ---------------------------------------------------------------------------
// Grid-wide deterministic reductions: every block writes one partial, the
// last block to arrive (ticket counter) sums the partials in block order and
// runs a scalar "finisher" on thread 0.
// ---------------------------------------------------------------------------
struct Scalars;
struct Slot {
  double* part;        // partials, >= total entries
  unsigned* ticket;    // arrival counter (reset to 0 by the last block)
  double* out;         // final sums
  int total;           // number of partials expected
  int op;              // finisher run by the last block (FIN_*)
  Scalars* sc;         // scalar state the finisher updates
  int base;            // inner-PCG state block (FIN_PCG_*)
  int flag;            // inner-PCG done flag index (FIN_PCG_*)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of `nv` values per thread; result valid in thread 0.
template <int NV_>
__device__ __forceinline__ void block_sum(double (&v)[NV_]) {
  __shared__ double sh[NV_][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV_; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV_; ++k) sh[k][wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV_; ++k) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
}

// Writes the block's NV_ partials at part[k*total + idx]; returns true on
// thread 0 of the last block, which then holds the final sums in v.
template <int NV_>
__device__ __forceinline__ bool slot_arrive(const Slot& s, int idx, double (&v)[NV_]) {
  block_sum<NV_>(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV_; ++k) s.part[(size_t)k * s.total + idx] = v[k];
    __threadfence();
    unsigned t = atomicAdd(s.ticket, 1u);
    last = (t == (unsigned)s.total - 1u);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // last block: sum partials in fixed order (all threads), result to thread 0
  double acc[NV_];
#pragma unroll
  for (int k = 0; k < NV_; ++k) {
    acc[k] = 0.0;
    for (int i = threadIdx.x; i < s.total; i += blockDim.x)
      acc[k] += ((volatile double*)s.part)[(size_t)k * s.total + i];
  }
  block_sum<NV_>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV_; ++k) v[k] = acc[k];
    *s.ticket = 0u;
  }
  return threadIdx.x == 0;
}

}  // namespace eth
#include "scalars.cuh"
namespace eth {

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
eth_status cuda_status(cudaError_t e, const char* what);

#define ETH_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::eth::cuda_status(e_, #call);         \
  } while (0)

#define ETH_TRY(call)                                                    \
  do {                                                                   \
    eth_status s_ = (call);                                              \
    if (s_ != ETH_OK) return s_;                                         \
  } while (0)

inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

// Dynamic shared memory above 48 KB is enabled per kernel AND per device
// (cudaFuncSetAttribute acts on the current device).  One SmemAttr per kernel
// records, per device, the largest size enabled so far; the first launch of
// that kernel on each device (and any larger request) sets the attribute.
constexpr int ETH_MAX_DEVICES = 64;
struct SmemAttr {
  std::atomic<int> bytes[ETH_MAX_DEVICES];
};
template <class K>
inline cudaError_t smem_attr(K kern, size_t bytes, SmemAttr& a) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < ETH_MAX_DEVICES;
  if (tracked && (int)bytes <= a.bytes[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess || !tracked) return e;
  int prev = a.bytes[dev].load(std::memory_order_relaxed);
  while (prev < (int)bytes && !a.bytes[dev].compare_exchange_weak(prev, (int)bytes)) {
  }
  return cudaSuccess;
}

// Makes a handle's device current for the duration of an entry point and
// restores the caller's device afterwards (all device memory and streams of a
// handle belong to the device that was current at its creation).
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    else if (err == cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
#define ETH_ON_DEVICE(g)                                                          \
  ::eth::DeviceGuard eth_dev_guard_((g)->dev);                                    \
  if (eth_dev_guard_.err != cudaSuccess) return ::eth::cuda_status(eth_dev_guard_.err, "cudaSetDevice")

}  // namespace eth
