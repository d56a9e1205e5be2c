// Shared device helpers: complex arithmetic on interleaved (re, im) pairs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace efie {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R> using cpx_t = typename C2<R>::T;

template <typename R>
__host__ __device__ __forceinline__ cpx_t<R> mk(R re, R im) {
  cpx_t<R> z;
  z.x = re;
  z.y = im;
  return z;
}
template <typename T>
__host__ __device__ __forceinline__ T cadd(T a, T b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename T>
__host__ __device__ __forceinline__ T csub(T a, T b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename T>
__host__ __device__ __forceinline__ T cmul(T a, T b) {
  T z;
  z.x = a.x * b.x - a.y * b.y;
  z.y = a.x * b.y + a.y * b.x;
  return z;
}
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(T& acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
template <typename T, typename S>
__host__ __device__ __forceinline__ T cscale(T a, S s) {
  a.x *= s;
  a.y *= s;
  return a;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Raises a kernel's dynamic shared-memory limit on the current device when a
// launch needs more than the limit set so far.  The limit is a per-device
// attribute; `done` keeps, per device (64 at most; later devices set it on
// every call), the largest value set.  Threads that race both set a value
// that covers their launch.
template <typename K>
inline void smem_attr_once(K kernel, int bytes, std::atomic<uint64_t>* done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  if (dev < 64 && done[dev].load(std::memory_order_acquire) >= (uint64_t)bytes) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess && dev < 64) {
    uint64_t cur = done[dev].load(std::memory_order_acquire);
    while (cur < (uint64_t)bytes && !done[dev].compare_exchange_weak(cur, (uint64_t)bytes)) {
    }
  }
}
// per-kernel state of smem_attr_once
struct SmemAttr {
  std::atomic<uint64_t> v[64];
  SmemAttr() {
    for (auto& x : v) x.store(0);
  }
};

}  // namespace efie
