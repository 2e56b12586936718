// Batched strided complex GEMM on CUDA cores (FP64 or FP32), the engine of
// the plain correlator path.
//
//   C[b](m, n) (+)= alpha * sum_k opA(A[b](m, k)) * B[b](k, n)
//
// Every operand index is mapped to a memory offset by a two-level affine
// map off(idx) = (idx / d0) * s1 + (idx % d0) * s0 (d0 = 0: off = idx * s0),
// and the batch index by a three-level split b = (b2 * n1 + b1) * n0 + b0
// with per-operand strides, so the mode contractions can read and write
// their tensors in place, whatever the index order.
#pragma once

#include "common.cuh"
#include "prof.cuh"

namespace distil {

struct Map2 {
  long long d0, s0, s1;
  __host__ __device__ __forceinline__ long long operator()(long long idx) const {
    return d0 ? (idx / d0) * s1 + (idx % d0) * s0 : idx * s0;
  }
};
inline Map2 map1(long long s0) { return Map2{0, s0, 0}; }
inline Map2 map2(long long d0, long long s0, long long s1) { return Map2{d0, s0, s1}; }

struct Batch3 {
  int n1, n0;                   // b = (b2 * n1 + b1) * n0 + b0
  long long a[3], b[3], c[3];   // strides of (b2, b1, b0) for A, B, C
};

template <typename T>
struct SimtGemmArgs {
  const Cx<T>* A;
  Map2 am, ak;
  const Cx<T>* B;
  Map2 bk, bn;
  Cx<T>* C;
  Map2 cm, cn;
  int M, N, K, batch;
  Batch3 bt;
  Cx<T> alpha;
  int accumulate;  // 1: C += alpha*AB, 0: C = alpha*AB
  int conjA;
};

constexpr int SG_TM = 64, SG_TN = 64, SG_TK = 16;

template <typename T>
__global__ void __launch_bounds__(256) simt_gemm_kernel(SimtGemmArgs<T> g) {
  __shared__ Cx<T> As[SG_TK][SG_TM + 1];
  __shared__ Cx<T> Bs[SG_TK][SG_TN + 1];
  __shared__ long long offA[SG_TM], offB[SG_TN];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * SG_TM, n0 = blockIdx.x * SG_TN;
  const int bidx = blockIdx.z;
  const int b0 = bidx % g.bt.n0;
  const int b1 = (bidx / g.bt.n0) % g.bt.n1;
  const int b2 = bidx / (g.bt.n0 * g.bt.n1);
  const Cx<T>* A = g.A + b2 * g.bt.a[0] + b1 * g.bt.a[1] + b0 * g.bt.a[2];
  const Cx<T>* B = g.B + b2 * g.bt.b[0] + b1 * g.bt.b[1] + b0 * g.bt.b[2];
  Cx<T>* C = g.C + b2 * g.bt.c[0] + b1 * g.bt.c[1] + b0 * g.bt.c[2];

  if (tid < SG_TM) offA[tid] = (m0 + tid < g.M) ? g.am(m0 + tid) : -1;
  else if (tid < SG_TM + SG_TN) offB[tid - SG_TM] = (n0 + tid - SG_TM < g.N) ? g.bn(n0 + tid - SG_TM) : -1;

  Cx<T> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cmake<T>(0, 0);
  __syncthreads();

  for (int k0 = 0; k0 < g.K; k0 += SG_TK) {
    // 64 x 16 elements of each operand, 4 per thread
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;
      int kk = e % SG_TK, mm = e / SG_TK;
      Cx<T> va = cmake<T>(0, 0);
      if (k0 + kk < g.K && offA[mm] >= 0) {
        va = A[offA[mm] + g.ak(k0 + kk)];
        if (g.conjA) va = cconj(va);
      }
      As[kk][mm] = va;
      Cx<T> vb = cmake<T>(0, 0);
      if (k0 + kk < g.K && offB[mm] >= 0) vb = B[g.bk(k0 + kk) + offB[mm]];
      Bs[kk][mm] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SG_TK; ++kk) {
      Cx<T> ra[4], rb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ra[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) rb[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], ra[a], rb[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int m = m0 + ty + 16 * a;
    if (m >= g.M) continue;
    long long om = g.cm(m);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int n = n0 + tx + 16 * b;
      if (n >= g.N) continue;
      Cx<T>* dst = C + om + g.cn(n);
      Cx<T> v = cmul(g.alpha, acc[a][b]);
      if (g.accumulate) v = cadd(v, *dst);
      *dst = v;
    }
  }
}

template <typename T>
int simt_gemm(distil_ctx* ctx, const SimtGemmArgs<T>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return DISTIL_OK;
  if (g.batch > 65535) {
    set_error("simt_gemm: batch %d too large", g.batch);
    return DISTIL_EINVAL;
  }
  dim3 grid((g.N + SG_TN - 1) / SG_TN, (g.M + SG_TM - 1) / SG_TM, g.batch);
  if (grid.y > 65535) {
    set_error("simt_gemm: M %d too large", g.M);
    return DISTIL_EINVAL;
  }
  {
    Launch L(ctx, sizeof(T) == 8 ? "simt_gemm_f64" : "simt_gemm_f32", s);
    simt_gemm_kernel<T><<<grid, 256, 0, s>>>(g);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

}  // namespace distil
