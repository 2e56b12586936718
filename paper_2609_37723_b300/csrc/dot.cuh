// Final contraction of the correlation matrix (FP64 accumulation):
//   C[q][a][b][t] += sum_terms coef sum_{i'<j', k} (V^a_{i'j'k} - V^a_{j'i'k}) X^{b,c}_{(i'j'),k}
// with V[a][slot][j'][i'][k] and X[b][c][pair][k] (correlate.cuh).  One block
// per (a, chunk of pairs); each thread keeps N_B FP64 partial sums, blocks
// reduce by warp shuffles and add into C with FP64 atomics.
#pragma once
#include "common.cuh"
#include "correlate.cuh"

namespace distil {

// C[q][a][b][t] += sum_terms coef sum_{i'<j',k} (V^a_{i'j'k} - V^a_{j'i'k}) X^{b,c}_{pair,k}
// V[a][slot][j'][i'][k], X[b][c][pair][k].  Block = (a, chunk of pairs).
template <typename T, int MAXB>
__global__ void __launch_bounds__(256)
dot_kernel(const Cx<T>* __restrict__ V, const Cx<T>* __restrict__ X, int nv, int nb,
           Cx<double>* __restrict__ C, long long cstride_a, long long cstride_b) {
  const int a = blockIdx.y;
  const long long P2 = comb2(nv);
  const long long n3 = (long long)nv * nv * nv;
  const long long work = P2 * nv;
  Cx<double> acc[MAXB];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) acc[b] = cmake(0.0, 0.0);
  const Cx<T>* Va = V + (long long)a * NPAIR * n3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < work;
       e += (long long)gridDim.x * blockDim.x) {
    long long q = e / nv;
    int k = (int)(e % nv);
    int ip, jp;
    pair_unrank(q, ip, jp);
    Cx<double> w[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const Cx<T>* Vs = Va + dot_slot(t) * n3;
      Cx<T> v1 = Vs[((long long)jp * nv + ip) * nv + k];  // V_{i'j'k}
      Cx<T> v2 = Vs[((long long)ip * nv + jp) * nv + k];  // V_{j'i'k}
      w[t] = cmake((double)v1.r - (double)v2.r, (double)v1.i - (double)v2.i);
      w[t] = cscale(w[t], dot_coef(t));
    }
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      if (b >= nb) break;
      const Cx<T>* Xb = X + (long long)b * NSRC * work;
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        Cx<T> x = Xb[dot_src(t) * work + e];
        cfma(acc[b], w[t], cmake((double)x.r, (double)x.i));
      }
    }
  }
  __shared__ Cx<double> red[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b = 0; b < nb && b < MAXB; ++b) {
    Cx<double> v = acc[b];
    for (int o = 16; o > 0; o >>= 1) {
      v.r += __shfl_xor_sync(0xffffffffu, v.r, o);
      v.i += __shfl_xor_sync(0xffffffffu, v.i, o);
    }
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      Cx<double> s = red[0];
      for (int u = 1; u < (int)(blockDim.x >> 5); ++u) s = cadd(s, red[u]);
      double* dst = reinterpret_cast<double*>(C + a * cstride_a + b * cstride_b);
      atomicAdd(dst, s.r);
      atomicAdd(dst + 1, s.i);
    }
    __syncthreads();
  }
}

}  // namespace distil
