// Plain (CUDA-core, FP64 or FP32) correlation matrix: the three mode
// contractions of correlate.cuh as batched strided GEMMs, one (t, p) at a
// time, then an FP64-accumulated dot over (i'<j', k).
#include "common.cuh"
#include "correlate.cuh"
#include "simt_gemm.cuh"
#include "prof.cuh"
#include "dot.cuh"

namespace distil {

// ------------------------------------------------------------------ glue
// G[a][k][j][i] = g_i g_j g_k Phi_ijk (dense antisymmetric, zero diagonal).
template <typename T>
__global__ void sink_dense_kernel(const Cx<T>* __restrict__ phi, const double* __restrict__ g, int nv, int nb,
                                  Cx<T>* __restrict__ G) {
  long long n3 = (long long)nv * nv * nv;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n3 * nb) return;
  int a = (int)(e / n3);
  long long r = e % n3;
  int i = (int)(r % nv), j = (int)((r / nv) % nv), k = (int)(r / ((long long)nv * nv));
  Cx<T> out = cmake<T>(0, 0);
  if (i != j && j != k && i != k) {
    int x = i, y = j, z = k, sgn = 1;
    // sort ascending, tracking the permutation parity
    if (x > y) { int tt = x; x = y; y = tt; sgn = -sgn; }
    if (y > z) { int tt = y; y = z; z = tt; sgn = -sgn; }
    if (x > y) { int tt = x; x = y; y = tt; sgn = -sgn; }
    const double* ga = g + (long long)a * nv;
    T w = (T)(ga[i] * ga[j] * ga[k] * sgn);
    out = cscale(phi[triple_rank(x, y, z)], w);
  }
  G[e] = out;
}

// S[b][pair(i'<j')][k'] = g_i' g_j' g_k' conj(Phi_{i'j'k'}).
template <typename T>
__global__ void source_pairs_kernel(const Cx<T>* __restrict__ phi, const double* __restrict__ g, int nv, int nb,
                                    Cx<T>* __restrict__ S) {
  long long P2 = comb2(nv);
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= P2 * nv * nb) return;
  int b = (int)(e / (P2 * nv));
  long long r = e % (P2 * nv);
  long long q = r / nv;
  int kp = (int)(r % nv);
  int ip, jp;
  pair_unrank(q, ip, jp);  // ip < jp
  Cx<T> out = cmake<T>(0, 0);
  if (kp != ip && kp != jp) {
    int x = ip, y = jp, z = kp, sgn = 1;
    if (y > z) { int tt = y; y = z; z = tt; sgn = -sgn; }
    if (x > y) { int tt = x; x = y; y = tt; sgn = -sgn; }
    const double* gb = g + (long long)b * nv;
    T w = (T)(gb[ip] * gb[jp] * gb[kp] * sgn);
    out = cscale(cconj(phi[triple_rank(x, y, z)]), w);
  }
  S[e] = out;
}

// Aa[a'][beta][i'][i] = Gamma_{alpha(beta) beta} tau[(alpha(beta) i)][(a' i')], a' < 3.
// Tc[c][k][k'] : c = 0: tau^{00}+tau^{11}; 1..4: tau^{02}, tau^{03}, tau^{12}, tau^{13}.
template <typename T>
__global__ void tau_blocks_kernel(const Cx<T>* __restrict__ tau, int nv, Cx<T>* __restrict__ Aa,
                                  Cx<T>* __restrict__ Tc) {
  long long n2 = (long long)nv * nv;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = 4LL * nv;
  if (e < 12 * n2) {
    int ap = (int)(e / (4 * n2));
    int beta = (int)((e / n2) % 4);
    int ipr = (int)((e / nv) % nv), i = (int)(e % nv);
    int alpha = beta ^ 1;
    T gam = (beta & 1) ? (T)-1 : (T)1;  // Gamma_{10}=+1, Gamma_{01}=-1, Gamma_{32}=+1, Gamma_{23}=-1
    Aa[e] = cscale(tau[(alpha * nv + i) * n4 + ap * nv + ipr], gam);
  } else if (e < 12 * n2 + 5 * n2) {
    long long f = e - 12 * n2;
    int c = (int)(f / n2);
    int k = (int)((f / nv) % nv), kp = (int)(f % nv);
    Cx<T> out;
    if (c == 0) {
      out = cadd(tau[(0 * nv + k) * n4 + 0 * nv + kp], tau[(1 * nv + k) * n4 + 1 * nv + kp]);
    } else {
      const int mu = (c <= 2) ? 0 : 1;
      const int gp = (c == 1 || c == 3) ? 2 : 3;
      out = tau[(mu * nv + k) * n4 + gp * nv + kp];
    }
    Tc[f] = out;
  }
}

// ------------------------------------------------------------- pipeline
template <typename T>
struct PlainWs {
  Cx<T> *G, *S, *Aa, *Tc, *U, *V, *X;
};

template <typename T>
static PlainWs<T> carve(Arena& ar, int nv, int nb) {
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv);
  PlainWs<T> w;
  w.G = ar.take<Cx<T>>(nb * n3);
  w.S = ar.take<Cx<T>>(nb * P2 * n);
  w.Aa = ar.take<Cx<T>>(12 * n2);
  w.Tc = ar.take<Cx<T>>(5 * n2);
  w.U = ar.take<Cx<T>>(nb * 12 * n3);
  w.V = ar.take<Cx<T>>(nb * NPAIR * n3);
  w.X = ar.take<Cx<T>>(nb * NSRC * P2 * n);
  return w;
}

size_t correlate_plain_workspace(int fp64, int nv, int nb) {
  Arena ar;
  if (fp64) carve<double>(ar, nv, nb);
  else carve<float>(ar, nv, nb);
  return ar.used + 256;
}

static inline unsigned nblk(long long work, int bs = 256) { return (unsigned)((work + bs - 1) / bs); }

template <typename T>
static int run_tp(distil_ctx* ctx, const Cx<T>* phi_snk_tp, const Cx<T>* phi_src_p, const Cx<T>* tau_t, const double* g_snk,
                  const double* g_src, int nv, int nb, const PlainWs<T>& w, Cx<double>* Cout,
                  long long cs_a, long long cs_b, cudaStream_t s) {
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv);
  {
    Launch L(ctx, "sink_dense", s);
    sink_dense_kernel<T><<<nblk(nb * n3), 256, 0, s>>>(phi_snk_tp, g_snk, nv, nb, w.G);
  }
  {
    Launch L(ctx, "source_pairs", s);
    source_pairs_kernel<T><<<nblk(nb * P2 * n), 256, 0, s>>>(phi_src_p, g_src, nv, nb, w.S);
  }
  {
    Launch L(ctx, "tau_blocks", s);
    tau_blocks_kernel<T><<<nblk(17 * n2), 256, 0, s>>>(tau_t, nv, w.Aa, w.Tc);
  }
  DISTIL_LAUNCH_CHECK();
  const Cx<T> one = cmake<T>(1, 0);

  // Step A: U[a][a'][i'][k][beta][j] = sum_i Aa[a'][beta][i'][i] G[a][k][j][i]
  {
    SimtGemmArgs<T> g{};
    g.A = w.Aa; g.am = map1(n); g.ak = map1(1);
    g.B = w.G; g.bk = map1(1); g.bn = map1(n);
    g.C = w.U; g.cm = map1(4 * n2); g.cn = map2(n, 1, 4 * n);
    g.M = nv; g.N = nv * nv; g.K = nv; g.batch = nb * 12;
    g.bt.n1 = 3; g.bt.n0 = 4;
    g.bt.a[0] = 0; g.bt.a[1] = 4 * n2; g.bt.a[2] = n2;
    g.bt.b[0] = n3; g.bt.b[1] = 0; g.bt.b[2] = 0;
    g.bt.c[0] = 12 * n3; g.bt.c[1] = 4 * n3; g.bt.c[2] = n;
    g.alpha = one; g.accumulate = 0; g.conjA = 0;
    DISTIL_TRY(simt_gemm(ctx, g, s));
  }
  // Step B: V[a][slot][j'][(i',k)] = sum_{(beta,j)} tau[(beta j)][(b' j')] U[a][a'][(i',k)][(beta,j)]
  const int slotbase[3] = {0, 3, 5};
  for (int ap = 0; ap < 3; ++ap) {
    SimtGemmArgs<T> g{};
    g.A = tau_t + (ap + 1) * n; g.am = map1(1); g.ak = map1(4 * n);
    g.B = w.U + ap * 4 * n3; g.bk = map1(1); g.bn = map1(4 * n);
    g.C = w.V + slotbase[ap] * n3; g.cm = map1(n2); g.cn = map1(1);
    g.M = (3 - ap) * nv; g.N = nv * nv; g.K = 4 * nv; g.batch = nb;
    g.bt.n1 = 1; g.bt.n0 = 1;
    g.bt.a[0] = 0; g.bt.b[0] = 12 * n3; g.bt.c[0] = NPAIR * n3;
    g.alpha = one; g.accumulate = 0; g.conjA = 0;
    DISTIL_TRY(simt_gemm(ctx, g, s));
  }
  // Source: X[b][c][pair][k] = sum_k' S[b][pair][k'] Tc[c][k][k']
  {
    SimtGemmArgs<T> g{};
    g.A = w.S; g.am = map1(n); g.ak = map1(1);
    g.B = w.Tc; g.bk = map1(1); g.bn = map1(n);
    g.C = w.X; g.cm = map1(n); g.cn = map1(1);
    g.M = (int)P2; g.N = nv; g.K = nv; g.batch = nb * NSRC;
    g.bt.n1 = 1; g.bt.n0 = NSRC;
    g.bt.a[0] = P2 * n; g.bt.a[1] = 0; g.bt.a[2] = 0;
    g.bt.b[0] = 0; g.bt.b[1] = 0; g.bt.b[2] = n2;
    g.bt.c[0] = NSRC * P2 * n; g.bt.c[1] = 0; g.bt.c[2] = P2 * n;
    g.alpha = one; g.accumulate = 0; g.conjA = 0;
    DISTIL_TRY(simt_gemm(ctx, g, s));
  }
  // Dot
  {
    long long work = P2 * n;
    unsigned gx = nblk(work);
    if (gx > 1024) gx = 1024;
    dim3 grid(gx, nb);
    Launch L(ctx, "dot", s);
    dot_kernel<T, 16><<<grid, 256, 0, s>>>(w.V, w.X, nv, nb, Cout, cs_a, cs_b);
    DISTIL_LAUNCH_CHECK();
  }
  return DISTIL_OK;
}

int correlate_plain(distil_ctx* ctx, int fp64, const void* phi_snk, const void* phi_src, const void* tau,
                    int nt, int nv, int np, const double* prof_snk, const double* prof_src, int prof_per_t, int nb,
                    void* C, int c_nt, int c_t0, void* ws, size_t ws_bytes, cudaStream_t s) {
  DISTIL_TRY(zero_c_columns(C, np * nb * nb, c_nt, c_t0, nt, s));
  if (nv < 3) return DISTIL_OK;
  const long long T3 = comb3(nv), n4 = 4LL * nv;
  Arena ar(ws, ws_bytes);
  Cx<double>* Cd = reinterpret_cast<Cx<double>*>(C);
  for (int t = 0; t < nt; ++t) {
    const double* g_snk = prof_snk + (prof_per_t ? (long long)t * nb * nv : 0);
    const double* g_src = prof_src;
    for (int q = 0; q < np; ++q) {
      Cx<double>* Cq = Cd + (long long)q * nb * nb * c_nt + c_t0 + t;
      if (fp64) {
        Arena a2 = ar;
        PlainWs<double> w = carve<double>(a2, nv, nb);
        if (!a2.fits()) { set_error("correlate: workspace too small"); return DISTIL_ENOMEM; }
        DISTIL_TRY(run_tp<double>(ctx, (const Cx<double>*)phi_snk + ((long long)t * np + q) * T3,
                                  (const Cx<double>*)phi_src + (long long)q * T3,
                                  (const Cx<double>*)tau + (long long)t * n4 * n4, g_snk, g_src, nv, nb, w,
                                  Cq, (long long)nb * c_nt, c_nt, s));
      } else {
        Arena a2 = ar;
        PlainWs<float> w = carve<float>(a2, nv, nb);
        if (!a2.fits()) { set_error("correlate: workspace too small"); return DISTIL_ENOMEM; }
        DISTIL_TRY(run_tp<float>(ctx, (const Cx<float>*)phi_snk + ((long long)t * np + q) * T3,
                                 (const Cx<float>*)phi_src + (long long)q * T3,
                                 (const Cx<float>*)tau + (long long)t * n4 * n4, g_snk, g_src, nv, nb, w,
                                 Cq, (long long)nb * c_nt, c_nt, s));
      }
    }
  }
  return DISTIL_OK;
}

}  // namespace distil
