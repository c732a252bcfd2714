// Device helpers shared by the spectau kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spectau.h"

namespace spectau {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };
template <typename T> using C = typename cplx<T>::t;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) {
  C<T> z; z.x = re; z.y = im; return z;
}
template <typename T> __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ C<T> cconj(C<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by i^q, q taken mod 4
template <typename T> __device__ __forceinline__ C<T> cipow(C<T> a, int q) {
  switch (q & 3) {
    case 0: return a;
    case 1: return mk<T>(-a.y, a.x);
    case 2: return mk<T>(-a.x, -a.y);
    default: return mk<T>(a.y, -a.x);
  }
}

// FP64 helpers that stay off the FP64 pipe (integer operations on the bit
// pattern): on GB300 each SM sub-partition retires only ~one FP64 warp
// instruction per 64 cycles, so sign flips and finiteness tests use the ALU.
__device__ __forceinline__ double dneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
__device__ __forceinline__ bool dfinite(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}
// floor(idx / n) for 0 <= idx < 2^20 from inv = 1/n in FP32: (idx + 1/2)/n
// lies at least 1/(2n) from an integer, and the two FP32 roundings (of inv
// and of the product, relative 2^-24 each) move it by under 2^-23 2^20/n =
// 2^-3/n, so the truncation is exact (a run-time integer division would
// cost a dozen instructions per element)
__device__ __forceinline__ int div_idx(int idx, float inv) { return (int)(((float)idx + 0.5f) * inv); }

// i^q * a for double2 without FP64 instructions
__device__ __forceinline__ double2 cipow_d(double2 a, int q) {
  switch (q & 3) {
    case 0: return a;
    case 1: return make_double2(dneg(a.y), a.x);
    case 2: return make_double2(dneg(a.x), dneg(a.y));
    default: return make_double2(a.y, dneg(a.x));
  }
}

// ---------------------------------------------------------------------------
// work items of a batched launch: one per CTA (queue null), or pulled from a
// device counter by a fixed, persistent grid (the work lists are sorted
// largest first, so the dynamic order balances uneven items)
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ void for_each_item(int nwork, int* queue, F&& body) {
  if (queue == nullptr) {
    body((int)blockIdx.x);
    return;
  }
  __shared__ int next_item;
  while (true) {
    if (threadIdx.x == 0) next_item = atomicAdd(queue, 1);
    __syncthreads();
    const int item = next_item;
    __syncthreads();                 // every thread has the item before thread 0 takes the next
    if (item >= nwork) break;
    body(item);
    __syncthreads();                 // the item's shared memory is free for the next one
  }
}

// ---------------------------------------------------------------------------
// device status word: first error wins; bad pencil recorded alongside
// ---------------------------------------------------------------------------
struct DevStatus {
  int code;            // 0 or a negative sp_status
  int pad;
  long long pencil;    // first failing pencil (or -1)
};

__device__ __forceinline__ void raise_status(DevStatus* st, int code, long long pencil) {
  if (atomicCAS(&st->code, 0, code) == 0) st->pencil = pencil;
}

}  // namespace spectau
