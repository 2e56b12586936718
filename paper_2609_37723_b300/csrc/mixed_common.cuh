// Pieces shared by the mixed-precision (split 16-bit, tensor-core) paths:
// split schemes, power-of-two operand scales, split/store helpers and the
// GEMM epilogues.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc.cuh"
#include "tc_host.cuh"

namespace distil {

// Products kept by each split scheme (piece of A, piece of B): all pairs
// whose piece orders add up to at most NP-1.
struct Scheme {
  bool bf16;
  int np;  // pieces per real value
  int nprod;
  int pa[6], pb[6];
};
inline Scheme scheme_of(int mode) {
  if (mode == DISTIL_MIXED_BF16X6) return Scheme{true, 3, 6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 2, 1, 0}};
  if (mode == DISTIL_MIXED_BF16X3) return Scheme{true, 2, 3, {0, 0, 1}, {0, 1, 0}};
  return Scheme{false, 2, 3, {0, 0, 1}, {0, 1, 0}};  // FP16X3
}

// --------------------------------------------------------------- scales
// A tensor with max |x| = m is stored as pieces of x * 2^e with
// e = 14 - ceil(log2 m), so the leading piece stays below 2^14 (FP16 range)
// and the trailing pieces stay normal for every entry within 2^-17 of m.
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  int e;
  frexpf(m, &e);  // m = f * 2^e, f in [0.5, 1)  ->  m <= 2^e
  return ldexpf(1.f, 14 - e);
}

// Max |x| of a complex array into *out (float bits, non-negative, so
// unsigned ordering is float ordering).  *out must start at 0.
template <typename T>
__global__ void maxabs_kernel(const Cx<T>* __restrict__ x, long long n, unsigned* out) {
  float m = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf((float)x[e].r), fabsf((float)x[e].i)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Store x (already scaled) as NP pieces into planes (piece*2 + ri).
template <bool BF16, int NP>
__device__ __forceinline__ void store_split(typename tc::Piece<BF16>::T* base, long long plane_stride, int ri,
                                            float x) {
  typename tc::Piece<BF16>::T p[NP];
  tc::split16<BF16, NP>(x, p);
#pragma unroll
  for (int i = 0; i < NP; ++i) base[(2 * i + ri) * plane_stride] = p[i];
}

// --------------------------------------------------------------- epilogues
// out[batch][row][col] = factor * D (complex FP32), two-level batch offset.
struct EpiC64 {
  float2* out;
  long long sb_hi, sb_lo;
  int b_lo;
  long long sr;
  int N;
  const float* factor;
  __device__ __forceinline__ void operator()(int batch, int row, int col0, const float* re, const float* im) const {
    const float f = *factor;
    float2* dst = out + (long long)(batch / b_lo) * sb_hi + (long long)(batch % b_lo) * sb_lo + (long long)row * sr +
                  col0;
    if (col0 + 16 <= N && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        d4[e] = make_float4(re[2 * e] * f, im[2 * e] * f, re[2 * e + 1] * f, im[2 * e + 1] * f);
    } else {
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (col0 + e < N) dst[e] = make_float2(re[e] * f, im[e] * f);
    }
  }
};

// Split epilogue: out planes (two-level batch) [plane][row][col] of NP pieces
// of factor * D; used where the result feeds the next tensor-core GEMM.
// Column c maps to (c / cdiv) * cs1 + (c % cdiv) * cs0 within the row.
template <bool BF16, int NP>
struct EpiSplit {
  typename tc::Piece<BF16>::T* out;
  long long sb_hi, sb_lo;
  int b_lo;
  long long plane_stride, sr;
  int cdiv;
  long long cs0, cs1;
  int N;
  const float* factor;
  __device__ __forceinline__ void operator()(int batch, int row, int col0, const float* re, const float* im) const {
    const float f = *factor;
    auto* base = out + (long long)(batch / b_lo) * sb_hi + (long long)(batch % b_lo) * sb_lo + (long long)row * sr;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      if (c >= N) break;
      auto* d = base + (long long)(c / cdiv) * cs1 + (long long)(c % cdiv) * cs0;
      store_split<BF16, NP>(d, plane_stride, 0, re[e] * f);
      store_split<BF16, NP>(d, plane_stride, 1, im[e] * f);
    }
  }
};

}  // namespace distil
