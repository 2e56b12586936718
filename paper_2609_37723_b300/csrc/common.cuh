// Shared device/host helpers of the distil library: complex arithmetic,
// error reporting, the context object and index bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "../../include/distil.h"

namespace distil {

// ---------------------------------------------------------------- complex
template <typename T>
struct alignas(2 * sizeof(T)) Cx {
  T r, i;
};

template <typename T>
__host__ __device__ __forceinline__ Cx<T> cmake(T r, T i) { Cx<T> z; z.r = r; z.i = i; return z; }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) { return cmake(a.r + b.r, a.i + b.i); }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) { return cmake(a.r - b.r, a.i - b.i); }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return cmake(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename T>
__host__ __device__ __forceinline__ Cx<T> cconj(Cx<T> a) { return cmake(a.r, -a.i); }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> cscale(Cx<T> a, T s) { return cmake(a.r * s, a.i * s); }
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(-a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i);
  acc.i = fma(a.i, b.r, acc.i);
}

// ---------------------------------------------------------------- triples
// Colex rank of i<j<k: C(k,3) + C(j,2) + i.
__host__ __device__ __forceinline__ long long comb2(long long n) { return n * (n - 1) / 2; }
__host__ __device__ __forceinline__ long long comb3(long long n) { return n * (n - 1) * (n - 2) / 6; }
__host__ __device__ __forceinline__ long long triple_rank(int i, int j, int k) {
  return comb3(k) + comb2(j) + i;
}
// Pair rank of j<k in colex order: C(k,2) + j; inverse by integer search.
__host__ __device__ __forceinline__ void pair_unrank(long long q, int& j, int& k) {
  int kk = (int)((1.0 + sqrt(1.0 + 8.0 * (double)q)) * 0.5);
  while (comb2(kk) > q) --kk;
  while (comb2(kk + 1) <= q) ++kk;
  k = kk;
  j = (int)(q - comb2(kk));
}

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
const char* get_error();

#define DISTIL_CHECK_ARG(cond, ...)         \
  do {                                      \
    if (!(cond)) {                          \
      ::distil::set_error(__VA_ARGS__);     \
      return DISTIL_EINVAL;                 \
    }                                       \
  } while (0)

#define DISTIL_CUDA(call)                                                              \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::distil::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e),      \
                          __FILE__, __LINE__);                                         \
      return DISTIL_ECUDA;                                                             \
    }                                                                                  \
  } while (0)

#define DISTIL_LAUNCH_CHECK()                                                          \
  do {                                                                                 \
    cudaError_t _e = cudaGetLastError();                                               \
    if (_e != cudaSuccess) {                                                           \
      ::distil::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e),  \
                          __FILE__, __LINE__);                                         \
      return DISTIL_ECUDA;                                                             \
    }                                                                                  \
  } while (0)

#define DISTIL_TRY(expr)           \
  do {                             \
    int _s = (expr);               \
    if (_s != DISTIL_OK) return _s;\
  } while (0)

inline bool is_mixed(int mode) {
  return mode == DISTIL_MIXED_BF16X6 || mode == DISTIL_MIXED_BF16X3 || mode == DISTIL_MIXED_FP16X3 ||
         mode == DISTIL_MIXED_FP16X6;
}
inline bool valid_mode(int mode) { return mode >= DISTIL_FP64 && mode <= DISTIL_MIXED_FP16X6; }

// Bump allocator over a caller-provided workspace (256-byte aligned slices).
struct Arena {
  char* base;
  size_t cap, used;
  explicit Arena(void* b = nullptr, size_t c = 0) : base((char*)b), cap(c), used(0) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    size_t bytes = count * sizeof(T);
    used = off + bytes;
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
  bool fits() const { return used <= cap; }
};

struct Profiler;
}  // namespace distil

// Opaque context (one per device).
struct distil_ctx {
  int device;
  int sm_count;
  int cc_major, cc_minor;
  unsigned int* d_error;   // device error word for bounded waits (0 = ok)
  distil::Profiler* prof;  // launch counts and optional event timing
  // tensor-core kernel variant of each mode-contraction site (step i,
  // step j, source): 0 = one 128 x 128 tile per CTA, 1 = persistent CTAs
  // with two 128 x 64 accumulator sets; set by distil_set_tuning or the
  // plan autotuner
  int tune[3];
  // limit of the tensor-core pipeline waits in SM clock cycles (0: the
  // default of about a second); distil_set_wait_limit
  long long wait_limit;
};
