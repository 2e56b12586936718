// Mixed-precision correlation matrix: the three mode contractions of
// correlate.cuh on tcgen05 tensor cores with operands split into 16-bit
// pieces (FP32 accumulation in TMEM), intermediates re-split by the GEMM
// epilogue, and the final dot accumulated in FP64.
//
// Per (t, p):
//   scales   power-of-two scales of tau, Phi_snk, Phi_src, the profiles
//   split    Aa (12 n x n), tauT (4n x 4n), Tc (5 n x n) from tau;
//            G[a] (n^2 x n) from Phi_snk and the profiles;
//            S[b] (P2 x n) from conj(Phi_src) and the profiles
//   step i   U[a][a'][(i',k)][(beta,j)] = sum_i Aa[a'beta][i'][i] G[a][(k,j)][i]
//   step j   V[a][slot][j'][(i',k)]     = sum_(beta,j) tauT[(b'j')][(beta j)] U[a][a'][(i',k)][(beta,j)]
//   source   X[b][c][pair][k]          = sum_k' S[b][pair][k'] Tc[c][k][k']
//   dot      C_ab                       (dot.cuh)
#include "correlate.cuh"
#include "dot.cuh"
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

using tc::Planes;

enum { SC_MTAU = 0, SC_MPHIS, SC_MPHI0, SC_MG, SC_STAU, SC_STC, SC_SG, SC_SS, SC_SU, SC_FA, SC_FB, SC_FX, SC_N };

__global__ void prof_max_kernel(const double* g, long long n, unsigned* out) {
  float m = 0.f;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) m = fmaxf(m, (float)fabs(g[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void scales_kernel(float* sc, int nv) {
  const float mt = __uint_as_float(reinterpret_cast<unsigned*>(sc)[SC_MTAU]);
  const float ms = __uint_as_float(reinterpret_cast<unsigned*>(sc)[SC_MPHIS]);
  const float m0 = __uint_as_float(reinterpret_cast<unsigned*>(sc)[SC_MPHI0]);
  const float mg = __uint_as_float(reinterpret_cast<unsigned*>(sc)[SC_MG]);
  const float g3 = mg * mg * mg;
  const float st = pow2_scale(mt), stc = pow2_scale(2.f * mt);
  const float sg = pow2_scale(ms * g3), ss = pow2_scale(m0 * g3);
  const float su = pow2_scale((float)nv * mt * ms * g3);
  sc[SC_STAU] = st;
  sc[SC_STC] = stc;
  sc[SC_SG] = sg;
  sc[SC_SS] = ss;
  sc[SC_SU] = su;
  sc[SC_FA] = su / (st * sg);
  sc[SC_FB] = 1.f / (st * su);
  sc[SC_FX] = 1.f / (ss * stc);
}

// Aa planes [12][NPL][n][ldn], tauT planes [NPL][4n][ld4], Tc planes [5][NPL][n][ldn].
template <bool BF16, int NP>
__global__ void split_tau_kernel(const float2* __restrict__ tau, int nv, const float* __restrict__ sc,
                                 typename tc::Piece<BF16>::T* __restrict__ Aa, long long ldn,
                                 typename tc::Piece<BF16>::T* __restrict__ TT, long long ld4,
                                 typename tc::Piece<BF16>::T* __restrict__ Tc) {
  constexpr int NPL = 2 * NP;
  const long long n = nv, n2 = n * n, n4 = 4 * n;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const float st = sc[SC_STAU], stc = sc[SC_STC];
  if (e < 12 * n2) {
    const int ab = (int)(e / n2);  // a'*4 + beta
    const int ap = ab / 4, beta = ab % 4, alpha = beta ^ 1;
    const int ipr = (int)((e / n) % n), i = (int)(e % n);
    const float gam = (beta & 1) ? -st : st;
    const float2 x = tau[(alpha * n + i) * n4 + ap * n + ipr];
    auto* d = Aa + (long long)ab * NPL * n * ldn + ipr * ldn + i;
    store_split<BF16, NP>(d, n * ldn, 0, x.x * gam);
    store_split<BF16, NP>(d, n * ldn, 1, x.y * gam);
  } else if (e < 28 * n2) {
    const long long f = e - 12 * n2;
    const long long r = f / n4, k = f % n4;  // tauT[r][k] = tau[k][r]
    const float2 x = tau[k * n4 + r];
    auto* d = TT + r * ld4 + k;
    store_split<BF16, NP>(d, n4 * ld4, 0, x.x * st);
    store_split<BF16, NP>(d, n4 * ld4, 1, x.y * st);
  } else if (e < 33 * n2) {
    const long long f = e - 28 * n2;
    const int c = (int)(f / n2);
    const int k = (int)((f / n) % n), kp = (int)(f % n);
    float2 x;
    if (c == 0) {
      const float2 a = tau[(0 * n + k) * n4 + 0 * n + kp], b = tau[(1 * n + k) * n4 + 1 * n + kp];
      x = make_float2(a.x + b.x, a.y + b.y);
    } else {
      const int mu = (c <= 2) ? 0 : 1;
      const int gp = (c == 1 || c == 3) ? 2 : 3;
      x = tau[(mu * n + k) * n4 + gp * n + kp];
    }
    auto* d = Tc + (long long)c * NPL * n * ldn + k * ldn + kp;
    store_split<BF16, NP>(d, n * ldn, 0, x.x * stc);
    store_split<BF16, NP>(d, n * ldn, 1, x.y * stc);
  }
}

// G planes [nb][NPL][n^2 rows (k,j)][ldn (i)] = s_G g_i g_j g_k Phi_ijk
template <bool BF16, int NP>
__global__ void split_sink_kernel(const float2* __restrict__ phi, const double* __restrict__ g, int nv, int nb,
                                  const float* __restrict__ sc, typename tc::Piece<BF16>::T* __restrict__ G,
                                  long long ldn) {
  constexpr int NPL = 2 * NP;
  const long long n = nv, n3 = n * n * n;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= nb * n3) return;
  const int a = (int)(e / n3);
  const long long r = e % n3;
  const int i = (int)(r % n), j = (int)((r / n) % n), k = (int)(r / (n * n));
  float2 v = make_float2(0.f, 0.f);
  if (i != j && j != k && i != k) {
    int x = i, y = j, z = k, sgn = 1;
    if (x > y) { int tt = x; x = y; y = tt; sgn = -sgn; }
    if (y > z) { int tt = y; y = z; z = tt; sgn = -sgn; }
    if (x > y) { int tt = x; x = y; y = tt; sgn = -sgn; }
    const double* ga = g + (long long)a * nv;
    const float w = (float)(ga[i] * ga[j] * ga[k] * sgn) * sc[SC_SG];
    const float2 p = phi[triple_rank(x, y, z)];
    v = make_float2(p.x * w, p.y * w);
  }
  auto* d = G + (long long)a * NPL * n * n * ldn + ((long long)k * n + j) * ldn + i;
  store_split<BF16, NP>(d, n * n * ldn, 0, v.x);
  store_split<BF16, NP>(d, n * n * ldn, 1, v.y);
}

// S planes [nb][NPL][P2 rows (i'<j')][ldn (k')] = s_S g g g conj(Phi_{i'j'k'})
template <bool BF16, int NP>
__global__ void split_source_kernel(const float2* __restrict__ phi, const double* __restrict__ g, int nv, int nb,
                                    const float* __restrict__ sc, typename tc::Piece<BF16>::T* __restrict__ S,
                                    long long ldn) {
  constexpr int NPL = 2 * NP;
  const long long n = nv, P2 = comb2(nv);
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= nb * P2 * n) return;
  const int b = (int)(e / (P2 * n));
  const long long r = e % (P2 * n);
  const long long q = r / n;
  const int kp = (int)(r % n);
  int ip, jp;
  pair_unrank(q, ip, jp);
  float2 v = make_float2(0.f, 0.f);
  if (kp != ip && kp != jp) {
    int x = ip, y = jp, z = kp, sgn = 1;
    if (y > z) { int tt = y; y = z; z = tt; sgn = -sgn; }
    if (x > y) { int tt = x; x = y; y = tt; sgn = -sgn; }
    const double* gb = g + (long long)b * nv;
    const float w = (float)(gb[ip] * gb[jp] * gb[kp] * sgn) * sc[SC_SS];
    const float2 p = phi[triple_rank(x, y, z)];
    v = make_float2(p.x * w, -p.y * w);
  }
  auto* d = S + (long long)b * NPL * P2 * ldn + q * ldn + kp;
  store_split<BF16, NP>(d, P2 * ldn, 0, v.x);
  store_split<BF16, NP>(d, P2 * ldn, 1, v.y);
}

// ------------------------------------------------------------------ workspace
struct MixedWs {
  float* sc;
  void *Aa, *TT, *Tc, *G, *S, *U;
  Cx<float>*V, *X;
  long long ldn, ld4;
};

static MixedWs carve_mixed(Arena& ar, int np_, int nv, int nb) {
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv);
  const int NPL = 2 * np_;
  MixedWs w;
  w.ldn = tc::pad64(n);
  w.ld4 = tc::pad64(4 * n);
  w.sc = ar.take<float>(64);
  w.Aa = ar.take<uint16_t>(12LL * NPL * n * w.ldn);
  w.TT = ar.take<uint16_t>((long long)NPL * 4 * n * w.ld4);
  w.Tc = ar.take<uint16_t>(5LL * NPL * n * w.ldn);
  w.G = ar.take<uint16_t>((long long)nb * NPL * n2 * w.ldn);
  w.S = ar.take<uint16_t>((long long)nb * NPL * P2 * w.ldn);
  w.U = ar.take<uint16_t>((long long)nb * 3 * NPL * n2 * w.ld4);
  w.V = ar.take<Cx<float>>((long long)nb * NPAIR * n3);
  w.X = ar.take<Cx<float>>((long long)nb * NSRC * P2 * n);
  return w;
}

size_t correlate_mixed_workspace(int mode, int nv, int nb) {
  Arena ar;
  carve_mixed(ar, scheme_of(mode).np, nv, nb);
  return ar.used + 256;
}

static inline unsigned nblk(long long work, int bs = 256) { return (unsigned)((work + bs - 1) / bs); }

template <bool BF16, int NP>
static int run_tp_mixed(distil_ctx* ctx, const Scheme& sch, const float2* phs, const float2* ph0, const float2* tau,
                        const double* g_snk, const double* g_src, int nv, int nb, const MixedWs& w,
                        Cx<double>* Cout, long long cs_a, long long cs_b, cudaStream_t s) {
  using P16 = typename tc::Piece<BF16>::T;
  constexpr int NPL = 2 * NP;
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv);
  // ---- scales
  DISTIL_CUDA(cudaMemsetAsync(w.sc, 0, 4 * sizeof(float), s));
  {
    Launch L(ctx, "maxabs", s);
    unsigned* u = reinterpret_cast<unsigned*>(w.sc);
    maxabs_kernel<float><<<64, 256, 0, s>>>((const Cx<float>*)tau, 16 * n2, u + SC_MTAU);
    maxabs_kernel<float><<<64, 256, 0, s>>>((const Cx<float>*)phs, comb3(nv), u + SC_MPHIS);
    maxabs_kernel<float><<<64, 256, 0, s>>>((const Cx<float>*)ph0, comb3(nv), u + SC_MPHI0);
    prof_max_kernel<<<1, 256, 0, s>>>(g_snk, (long long)nb * nv, u + SC_MG);
    if (g_src != g_snk) prof_max_kernel<<<1, 256, 0, s>>>(g_src, (long long)nb * nv, u + SC_MG);
    scales_kernel<<<1, 1, 0, s>>>(w.sc, nv);
  }
  // ---- split operands
  {
    Launch L(ctx, "split_operands", s);
    split_tau_kernel<BF16, NP><<<nblk(33 * n2), 256, 0, s>>>(tau, nv, w.sc, (P16*)w.Aa, w.ldn, (P16*)w.TT, w.ld4,
                                                             (P16*)w.Tc);
    split_sink_kernel<BF16, NP><<<nblk(nb * n3), 256, 0, s>>>(phs, g_snk, nv, nb, w.sc, (P16*)w.G, w.ldn);
    split_source_kernel<BF16, NP><<<nblk(nb * P2 * n), 256, 0, s>>>(ph0, g_src, nv, nb, w.sc, (P16*)w.S, w.ldn);
  }
  DISTIL_LAUNCH_CHECK();
  tc::GemmCfg cfg{};
  cfg.nprod = sch.nprod;
  for (int i = 0; i < sch.nprod; ++i) {
    cfg.pa[i] = sch.pa[i];
    cfg.pb[i] = sch.pb[i];
  }
  cfg.err = ctx->d_error;
  // KC / stages per scheme
  constexpr int KC = NP == 2 ? 32 : 16;
  constexpr int ST256 = NP == 2 ? 2 : 3;
  constexpr int ST128 = NP == 2 ? 3 : 4;

  // ---- step i: batch (a, a'beta) = nb x 12
  {
    Planes A{w.Aa, n, n, NPL, 12, w.ldn, n * w.ldn, NPL * n * w.ldn};
    Planes B{w.G, n, n2, NPL, nb, w.ldn, n2 * w.ldn, NPL * n2 * w.ldn};
    cfg.M = nv; cfg.N = (int)n2; cfg.K = nv;
    cfg.a = tc::OpMap{1, 12, 1, 0, 0};
    cfg.b = tc::OpMap{12, nb, 1, 0, 0};
    EpiSplit<BF16, NP> epi;
    epi.out = (P16*)w.U;
    epi.b_lo = 4;
    epi.sb_hi = (long long)NPL * n2 * w.ld4;  // (a, a') block
    epi.sb_lo = n;                            // beta -> column offset
    epi.plane_stride = n2 * w.ld4;
    epi.sr = n * w.ld4;                       // i' -> rows (i', k)
    epi.cdiv = nv; epi.cs1 = w.ld4; epi.cs0 = 1;
    epi.N = (int)n2;
    epi.factor = w.sc + SC_FA;
    DISTIL_TRY((tc::launch_gemm<256, KC, NPL, ST256, BF16>(ctx, "tc_gemm_step_i", A, B, cfg, nb * 12, epi, s)));
  }
  // ---- step j: per a' (rows b' > a'), batch a
  const int slotbase[3] = {0, 3, 5};
  for (int ap = 0; ap < 3; ++ap) {
    Planes A{w.TT, 4 * n, 4 * n, NPL, 1, w.ld4, 4 * n * w.ld4, NPL * 4 * n * w.ld4};
    Planes B{w.U, 4 * n, n2, NPL, 3LL * nb, w.ld4, n2 * w.ld4, NPL * n2 * w.ld4};
    cfg.M = (3 - ap) * nv; cfg.N = (int)n2; cfg.K = 4 * nv;
    cfg.a = tc::OpMap{1, 1, 0, 0, (ap + 1) * nv};
    cfg.b = tc::OpMap{1, nb, 3, ap, 0};
    EpiC64 epi;
    epi.out = reinterpret_cast<float2*>(w.V + (long long)slotbase[ap] * n3);
    epi.b_lo = 1; epi.sb_hi = NPAIR * n3; epi.sb_lo = 0;
    epi.sr = n2; epi.N = (int)n2;
    epi.factor = w.sc + SC_FB;
    DISTIL_TRY((tc::launch_gemm<256, KC, NPL, ST256, BF16>(ctx, "tc_gemm_step_j", A, B, cfg, nb, epi, s)));
  }
  // ---- source: batch (b, c) = nb x 5
  {
    Planes A{w.S, n, P2, NPL, nb, w.ldn, P2 * w.ldn, NPL * P2 * w.ldn};
    Planes B{w.Tc, n, n, NPL, NSRC, w.ldn, n * w.ldn, NPL * n * w.ldn};
    cfg.M = (int)P2; cfg.N = nv; cfg.K = nv;
    cfg.a = tc::OpMap{NSRC, nb, 1, 0, 0};
    cfg.b = tc::OpMap{1, NSRC, 1, 0, 0};
    EpiC64 epi;
    epi.out = reinterpret_cast<float2*>(w.X);
    epi.b_lo = 1; epi.sb_hi = P2 * n; epi.sb_lo = 0;
    epi.sr = n; epi.N = nv;
    epi.factor = w.sc + SC_FX;
    if (nv > 64)
      DISTIL_TRY((tc::launch_gemm<128, KC, NPL, ST128, BF16>(ctx, "tc_gemm_source", A, B, cfg, nb * NSRC, epi, s)));
    else
      DISTIL_TRY((tc::launch_gemm<64, KC, NPL, ST128, BF16>(ctx, "tc_gemm_source", A, B, cfg, nb * NSRC, epi, s)));
  }
  // ---- dot
  {
    long long work = P2 * n;
    unsigned gx = nblk(work);
    if (gx > 1024) gx = 1024;
    Launch L(ctx, "dot", s);
    dot_kernel<float, 16><<<dim3(gx, nb), 256, 0, s>>>(w.V, w.X, nv, nb, Cout, cs_a, cs_b);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

int mixed_mode_built(int mode) { return is_mixed(mode) ? 1 : 0; }

int correlate_mixed(distil_ctx* ctx, int mode, const void* phi_snk, const void* phi_src, const void* tau, int nt,
                    int nv, int np, const double* prof, int nb, int prof_per_t, void* C, void* ws,
                    size_t ws_bytes, cudaStream_t s) {
  DISTIL_CUDA(cudaMemsetAsync(C, 0, sizeof(Cx<double>) * (size_t)np * nb * nb * nt, s));
  if (nv < 3) return DISTIL_OK;
  const Scheme sch = scheme_of(mode);
  Arena ar(ws, ws_bytes);
  MixedWs w = carve_mixed(ar, sch.np, nv, nb);
  if (!ar.fits()) {
    set_error("correlate: workspace too small");
    return DISTIL_ENOMEM;
  }
  const long long T3 = comb3(nv), n4 = 4LL * nv;
  Cx<double>* Cd = reinterpret_cast<Cx<double>*>(C);
  for (int t = 0; t < nt; ++t) {
    const double* g_snk = prof + (prof_per_t ? (long long)t * nb * nv : 0);
    for (int q = 0; q < np; ++q) {
      const float2* phs = (const float2*)phi_snk + ((long long)t * np + q) * T3;
      const float2* ph0 = (const float2*)phi_src + (long long)q * T3;
      const float2* ta = (const float2*)tau + (long long)t * n4 * n4;
      Cx<double>* Cq = Cd + (long long)q * nb * nb * nt + t;
      int st;
      if (mode == DISTIL_MIXED_BF16X6)
        st = run_tp_mixed<true, 3>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, (long long)nb * nt, nt, s);
      else if (mode == DISTIL_MIXED_BF16X3)
        st = run_tp_mixed<true, 2>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, (long long)nb * nt, nt, s);
      else
        st = run_tp_mixed<false, 2>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, (long long)nb * nt, nt, s);
      if (st != DISTIL_OK) return st;
    }
  }
  return DISTIL_OK;
}

}  // namespace distil
