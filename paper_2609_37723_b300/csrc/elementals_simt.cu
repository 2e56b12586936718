// Plain (CUDA-core) nucleon elementals, FP64 or FP32.
//
//   Phi[t][q]_ijk = sum_s exp(-i p_q.x_s) sum_a v_i^a(s) w_jk^a(s),
//   w_jk(s) = v_j(s) x v_k(s)   (eps_abc v_j^b v_k^c, the colour cross product)
//
// i.e. the elementals of Sec. 2.1 as one momentum-projected contraction
// over (site, colour) of E_(q,i) = exp(-ip.x) v_i against the cross products
// of the pairs j<k.  Each CTA owns a 64 (q,i) x 64 pair tile of one
// timeslice, stages 6 sites of E and w in shared memory per step and keeps
// a 4x4 complex micro-tile per thread.  Only i < j outputs are stored;
// tiles with no i < j are skipped.
#include "common.cuh"
#include "elementals.cuh"
#include "prof.cuh"

namespace distil {

constexpr int EL_TILE = 64;
constexpr int EL_KS = 6;  // sites per shared-memory step

template <typename T>
__global__ void __launch_bounds__(256)
elementals_simt_kernel(const Cx<T>* __restrict__ v, int V3, int nv, int np,
                       Cx<T>* __restrict__ phi, long long T3, long long P2, ElemParams<T> prm) {
  __shared__ Cx<T> Es[EL_KS * 3][EL_TILE + 1];
  __shared__ Cx<T> Ws[EL_KS * 3][EL_TILE + 1];
  __shared__ int rp[EL_TILE], ri[EL_TILE], pj[EL_TILE], pk[EL_TILE];
  __shared__ int s_imin, s_jmax;

  const int tid = threadIdx.x;
  const int t = blockIdx.z;
  const long long q0 = (long long)blockIdx.x * EL_TILE;
  const int r0 = blockIdx.y * EL_TILE;
  const int L = prm.L;
  if (tid == 0) { s_imin = 1 << 30; s_jmax = -1; }
  __syncthreads();
  if (tid < EL_TILE) {
    int r = r0 + tid;
    if (r < np * nv) {
      rp[tid] = r / nv;
      ri[tid] = r % nv;
      atomicMin(&s_imin, ri[tid]);
    } else {
      rp[tid] = -1; ri[tid] = 0;
    }
  } else if (tid < 2 * EL_TILE) {
    int c = tid - EL_TILE;
    long long q = q0 + c;
    if (q < P2) {
      int j, k;
      pair_unrank(q, j, k);
      pj[c] = j; pk[c] = k;
      atomicMax(&s_jmax, j);
    } else {
      pj[c] = -1; pk[c] = -1;
    }
  }
  __syncthreads();
  if (s_imin >= s_jmax) return;  // no i < j in this tile

  const Cx<T>* vt = v + (long long)t * nv * V3 * 3;
  const int tx = tid % 16, ty = tid / 16;
  Cx<T> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cmake<T>(0, 0);

  for (int s0 = 0; s0 < V3; s0 += EL_KS) {
    // E: 64 rows x EL_KS sites, W: 64 pairs x EL_KS sites
    for (int e = tid; e < EL_TILE * EL_KS; e += 256) {
      int sl = e % EL_KS, idx = e / EL_KS;
      int s = s0 + sl;
      // ---- E
      Cx<T> e0 = cmake<T>(0, 0), e1 = e0, e2 = e0;
      if (s < V3 && rp[idx] >= 0) {
        int x = s % L, y = (s / L) % L, z = s / (L * L);
        int p = rp[idx];
        int m = (prm.mom[p][0] * x + prm.mom[p][1] * y + prm.mom[p][2] * z) % L;
        if (m < 0) m += L;
        Cx<T> ph = prm.ptab[m];
        const Cx<T>* src = vt + ((long long)ri[idx] * V3 + s) * 3;
        e0 = cmul(ph, src[0]); e1 = cmul(ph, src[1]); e2 = cmul(ph, src[2]);
      }
      Es[sl * 3 + 0][idx] = e0; Es[sl * 3 + 1][idx] = e1; Es[sl * 3 + 2][idx] = e2;
      // ---- W
      Cx<T> w0 = cmake<T>(0, 0), w1 = w0, w2 = w0;
      if (s < V3 && pj[idx] >= 0) {
        const Cx<T>* a = vt + ((long long)pj[idx] * V3 + s) * 3;
        const Cx<T>* b = vt + ((long long)pk[idx] * V3 + s) * 3;
        Cx<T> a0 = a[0], a1 = a[1], a2 = a[2], b0 = b[0], b1 = b[1], b2 = b[2];
        w0 = csub(cmul(a1, b2), cmul(a2, b1));
        w1 = csub(cmul(a2, b0), cmul(a0, b2));
        w2 = csub(cmul(a0, b1), cmul(a1, b0));
      }
      Ws[sl * 3 + 0][idx] = w0; Ws[sl * 3 + 1][idx] = w1; Ws[sl * 3 + 2][idx] = w2;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < EL_KS * 3; ++kk) {
      Cx<T> ra[4], rb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ra[a] = Es[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) rb[b] = Ws[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], ra[a], rb[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int rr = ty + 16 * a;
    if (rp[rr] < 0) continue;
    int i = ri[rr];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int cc = tx + 16 * b;
      int j = pj[cc];
      if (j < 0 || i >= j) continue;
      phi[((long long)t * np + rp[rr]) * T3 + triple_rank(i, j, pk[cc])] = acc[a][b];
    }
  }
}

template <typename T>
int elementals_simt(distil_ctx* ctx, const Cx<T>* v, int L, int nt, int nv, const int32_t* mom, int np, Cx<T>* phi,
                    cudaStream_t stream) {
  const long long T3 = comb3(nv), P2 = comb2(nv);
  const int V3 = L * L * L;
  if (T3 == 0) return DISTIL_OK;
  ElemParams<T> prm;
  fill_elem_params(prm, L, mom, np);
  dim3 grid((unsigned)((P2 + EL_TILE - 1) / EL_TILE), (np * nv + EL_TILE - 1) / EL_TILE, nt);
  if (grid.y > 65535 || grid.z > 65535) {
    set_error("elementals: grid too large (np*nv=%d, nt=%d)", np * nv, nt);
    return DISTIL_EINVAL;
  }
  {
    Launch Lz(ctx, sizeof(T) == 8 ? "elementals_simt_f64" : "elementals_simt_f32", stream);
    elementals_simt_kernel<T><<<grid, 256, 0, stream>>>(v, V3, nv, np, phi, T3, P2, prm);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

template int elementals_simt<double>(distil_ctx*, const Cx<double>*, int, int, int, const int32_t*, int, Cx<double>*, cudaStream_t);
template int elementals_simt<float>(distil_ctx*, const Cx<float>*, int, int, int, const int32_t*, int, Cx<float>*, cudaStream_t);

}  // namespace distil
