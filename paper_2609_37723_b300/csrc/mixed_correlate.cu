// Mixed-precision correlation matrix: the three mode contractions of
// correlate.cuh on tcgen05 tensor cores with operands split into 16-bit
// pieces with per-row power-of-two exponents (mixed_common.cuh), FP32
// accumulation in TMEM combined in FP64, FP64 intermediates between the
// contractions, and the final dot accumulated in FP64.
//
// Per (t, p):
//   split    Aa  rows (a'beta, i')  K i        from Gamma_beta tau[(alpha(beta) i)][(a' i')]
//            tauT rows (b' j')      K (beta j) from tau[(beta j)][(b' j')]
//            Tc  rows (c, k)        K k'       from the five source blocks
//            G   rows (a, (k,j))    K i        from g g g Phi_snk
//            S   rows (b, i'<j')    K k'       from g g g conj(Phi_src)
//   step i   U[a][a'][(i',k)][(beta,j)] = sum_i Aa G, split by the epilogue
//            with the row exponent of the Cauchy-Schwarz bound
//            |U| <= max_beta |Aa row| * max_j |G row|
//   step j   V[a][slot][j'][(i',k)]     = sum_(beta,j) U tauT        (complex128)
//   source   X[b][c][pair][k]           = sum_k' S Tc                (complex128)
//   dot      C_ab                         (dot.cuh)
#include "correlate.cuh"
#include "dot.cuh"
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

using tc::Planes;

// ------------------------------------------------------------------ sources
__device__ __forceinline__ double2 d2(float2 x) { return make_double2(x.x, x.y); }

struct AaSrc {  // rows (a'*4 + beta)*n + i', K = i
  const float2* tau;
  int n;
  __device__ __forceinline__ double2 operator()(long long r, int i) const {
    const int ab = (int)(r / n), ip = (int)(r % n);
    const int ap = ab >> 2, beta = ab & 3, alpha = beta ^ 1;
    const float2 x = tau[((long long)alpha * n + i) * 4 * n + ap * n + ip];
    // Gamma_{10} = Gamma_{32} = +1, Gamma_{01} = Gamma_{23} = -1
    return (beta & 1) ? make_double2(-x.x, -x.y) : d2(x);
  }
};
struct TTSrc {  // rows (b'j'), K = (beta j): tau^T
  const float2* tau;
  int n;
  __device__ __forceinline__ double2 operator()(long long r, int k) const {
    return d2(tau[(long long)k * 4 * n + r]);
  }
};
struct TcSrc {  // rows c*n + k, K = k': T^c[k][k']
  const float2* tau;
  int n;
  __device__ __forceinline__ double2 operator()(long long r, int kp) const {
    const int c = (int)(r / n), k = (int)(r % n);
    const long long n4 = 4LL * n;
    if (c == 0) {
      const float2 a = tau[(long long)k * n4 + kp], b = tau[((long long)n + k) * n4 + n + kp];
      return make_double2((double)a.x + b.x, (double)a.y + b.y);
    }
    const int mu = (c <= 2) ? 0 : 1;
    const int gp = (c == 1 || c == 3) ? 2 : 3;
    return d2(tau[((long long)mu * n + k) * n4 + gp * n + kp]);
  }
};
// sorted-triple lookup with sign; 0 on a repeated index
__device__ __forceinline__ double2 phi_at(const double2* phi, int i, int j, int k, double w) {
  if (i == j || j == k || i == k) return make_double2(0.0, 0.0);
  int x = i, y = j, z = k;
  if (x > y) { int t = x; x = y; y = t; w = -w; }
  if (y > z) { int t = y; y = z; z = t; w = -w; }
  if (x > y) { int t = x; x = y; y = t; w = -w; }
  const double2 p = phi[triple_rank(x, y, z)];
  return make_double2(p.x * w, p.y * w);
}
struct GSrc {  // rows a*n^2 + k*n + j, K = i: g_i g_j g_k Phi_ijk
  const double2* phi;
  const double* g;
  int n;
  __device__ __forceinline__ double2 operator()(long long r, int i) const {
    const long long n2 = (long long)n * n;
    const int a = (int)(r / n2);
    const int k = (int)((r % n2) / n), j = (int)(r % n);
    const double* ga = g + (long long)a * n;
    return phi_at(phi, i, j, k, ga[i] * ga[j] * ga[k]);
  }
};
struct SSrc {  // rows b*P2 + pair(i'<j'), K = k': g g g conj(Phi_{i'j'k'})
  const double2* phi;
  const double* g;
  int n;
  long long P2;
  __device__ __forceinline__ double2 operator()(long long r, int kp) const {
    const int b = (int)(r / P2);
    int ip, jp;
    pair_unrank(r % P2, ip, jp);
    const double* gb = g + (long long)b * n;
    const double2 v = phi_at(phi, ip, jp, kp, gb[ip] * gb[jp] * gb[kp]);
    return make_double2(v.x, -v.y);
  }
};

// eU[(a*3 + a')*n^2 + i'*n + k] = exponent of max_beta |Aa row (a'beta, i')| * max_j |G row (a, k, j)|
__global__ void u_exponent_kernel(const float* __restrict__ nAa, const float* __restrict__ nG, int n, int nb,
                                  int* __restrict__ eU) {
  const long long n2 = (long long)n * n;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= 3LL * nb * n2) return;
  const int ab = (int)(e / n2);  // a*3 + a'
  const int a = ab / 3, ap = ab % 3;
  const int ip = (int)((e % n2) / n), k = (int)(e % n);
  float mA = 0.f;
  for (int beta = 0; beta < 4; ++beta) mA = fmaxf(mA, nAa[(ap * 4 + beta) * n + ip]);
  float mG = 0.f;
  const float* g = nG + (long long)a * n2 + (long long)k * n;
  for (int j = 0; j < n; ++j) mG = fmaxf(mG, g[j]);
  eU[e] = row_exponent_d((double)mA * (double)mG * (1.0 + 1e-5));
}

// Step i epilogue: split U straight from the FP64-combined accumulators into
// the A-operand pieces of step j, U[(a,a')][plane][(i',k)][(beta,j)].
template <bool BF16, bool FIXED, int NPC>
struct EpiSplitU {
  typename tc::Piece<BF16>::T* out;
  const int* eU;
  int n, H;
  long long ld4;
  __device__ __forceinline__ bool skip_tile(int, int, int) const { return false; }
  __device__ __forceinline__ void operator()(int batch, int row, int col0, const double* re,
                                             const double* im) const {
    const long long n2 = (long long)n * n;
    const int aa = batch >> 2, beta = batch & 3;  // aa = a*3 + a'
    const long long ps = n2 * ld4;
    auto* base = out + (long long)aa * (2 * NPC) * ps;
#pragma unroll 4
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      if (c >= (int)n2) break;
      const int k = c / n, j = c % n;
      const long long ur = (long long)row * n + k;
      const int ex = eU[(long long)aa * n2 + ur];
      typename tc::Piece<BF16>::T pr[NPC], pi[NPC];
      make_pieces<BF16, FIXED, NPC>(re[e], ex, H, pr);
      make_pieces<BF16, FIXED, NPC>(im[e], ex, H, pi);
      auto* d = base + ur * ld4 + (long long)beta * n + j;
#pragma unroll
      for (int q = 0; q < NPC; ++q) {
        d[(2 * q) * ps] = pr[q];
        d[(2 * q + 1) * ps] = pi[q];
      }
    }
  }
};

// ------------------------------------------------------------------ workspace
struct MixedWs {
  void *Aa, *TT, *Tc, *G, *S, *U;
  int *eAa, *eTT, *eTc, *eG, *eS, *eU;
  float *nAa, *nG;
  Cx<double>*V, *X;
  long long ldn, ld4;
};

static MixedWs carve_mixed(Arena& ar, const Scheme& sc, int nv, int nb) {
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv);
  const int npa = 2 * sc.na, npb = 2 * sc.nb;
  MixedWs w;
  w.ldn = tc::pad64(n);
  w.ld4 = tc::pad64(4 * n);
  w.Aa = ar.take<uint16_t>(12LL * npa * n * w.ldn);
  w.TT = ar.take<uint16_t>((long long)npb * 4 * n * w.ld4);
  w.Tc = ar.take<uint16_t>(5LL * npb * n * w.ldn);
  w.G = ar.take<uint16_t>((long long)nb * npb * n2 * w.ldn);
  w.S = ar.take<uint16_t>((long long)nb * npa * P2 * w.ldn);
  w.U = ar.take<uint16_t>((long long)nb * 3 * npa * n2 * w.ld4);
  w.eAa = ar.take<int>(12 * n);
  w.eTT = ar.take<int>(4 * n);
  w.eTc = ar.take<int>(5 * n);
  w.eG = ar.take<int>(nb * n2);
  w.eS = ar.take<int>(nb * P2);
  w.eU = ar.take<int>(3 * nb * n2);
  w.nAa = ar.take<float>(12 * n);
  w.nG = ar.take<float>(nb * n2);
  w.V = ar.take<Cx<double>>((long long)nb * NPAIR * n3);
  w.X = ar.take<Cx<double>>((long long)nb * NSRC * P2 * n);
  return w;
}

size_t correlate_mixed_workspace(int mode, int nv, int nb) {
  Arena ar;
  carve_mixed(ar, scheme_of(mode), nv, nb);
  return ar.used + 256;
}

// GEMM with the N tile chosen from N (TMEM holds 4 x NT columns).
template <bool BF16, int NPLA, int NPLB, class Epi>
static int gemm(distil_ctx* ctx, const char* name, const Planes& A, const Planes& B, const tc::GemmCfg& cfg,
                int batch, const Epi& epi, cudaStream_t s) {
  constexpr int KC = 32;
  constexpr int ST128 = (NPLA + NPLB) > 8 ? 2 : 3;
  if (cfg.N > 64)
    return tc::launch_gemm<128, KC, NPLA, NPLB, ST128, BF16>(ctx, name, A, B, cfg, batch, epi, s);
  if (cfg.N > 32) return tc::launch_gemm<64, KC, NPLA, NPLB, 2, BF16>(ctx, name, A, B, cfg, batch, epi, s);
  return tc::launch_gemm<32, KC, NPLA, NPLB, 2, BF16>(ctx, name, A, B, cfg, batch, epi, s);
}

template <bool BF16, bool FIXED, int NA, int NB>
static int run_tp_mixed(distil_ctx* ctx, const Scheme& sch, const double2* phs, const double2* ph0,
                        const float2* tau, const double* g_snk, const double* g_src, int nv, int nb,
                        const MixedWs& w, Cx<double>* Cout, long long cs_a, long long cs_b, cudaStream_t s) {
  constexpr int NPLA = 2 * NA, NPLB = 2 * NB;
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv);
  using P16 = typename tc::Piece<BF16>::T;
  // ---- split operands (one warp per row, per-row exponents)
  DISTIL_TRY((split_rows<BF16, FIXED, NA>(ctx, AaSrc{tau, nv}, 12 * n, n, nv, sch.H, w.Aa, w.ldn, w.eAa, s, w.nAa)));
  DISTIL_TRY((split_rows<BF16, FIXED, NB>(ctx, TTSrc{tau, nv}, 4 * n, 4 * n, 4 * nv, sch.H, w.TT, w.ld4, w.eTT, s)));
  DISTIL_TRY((split_rows<BF16, FIXED, NB>(ctx, TcSrc{tau, nv}, 5 * n, n, nv, sch.H, w.Tc, w.ldn, w.eTc, s)));
  DISTIL_TRY((split_rows<BF16, FIXED, NB>(ctx, GSrc{phs, g_snk, nv}, nb * n2, n2, nv, sch.H, w.G, w.ldn, w.eG, s, w.nG)));
  DISTIL_TRY((split_rows<BF16, FIXED, NA>(ctx, SSrc{ph0, g_src, nv, P2}, nb * P2, P2, nv, sch.H, w.S, w.ldn, w.eS, s)));
  {
    Launch L(ctx, "u_exponent", s);
    u_exponent_kernel<<<(unsigned)((3 * nb * n2 + 255) / 256), 256, 0, s>>>(w.nAa, w.nG, nv, nb, w.eU);
  }
  DISTIL_LAUNCH_CHECK();

  tc::GemmCfg cfg{};
  fill_products(cfg, sch);
  cfg.err = ctx->d_error;

  // ---- step i: batch (a, a'beta) = nb x 12, output split into U pieces
  {
    Planes A = planes_of(w.Aa, n, n, 12, NPLA, w.ldn);
    Planes B = planes_of(w.G, n, n2, nb, NPLB, w.ldn);
    cfg.M = nv; cfg.N = (int)n2; cfg.K = nv;
    cfg.a = tc::OpMap{1, 12, 1, 0, 0, nv, w.eAa};
    cfg.b = tc::OpMap{12, nb, 1, 0, 0, (int)n2, w.eG};
    EpiSplitU<BF16, FIXED, NA> epi{(P16*)w.U, w.eU, nv, sch.H, w.ld4};
    DISTIL_TRY((gemm<BF16, NPLA, NPLB>(ctx, "tc_gemm_step_i", A, B, cfg, nb * 12, epi, s)));
  }
  // ---- step j: per a' (rows b' > a'), batch a; V[a][slot][j'][(i',k)]
  const int slotbase[3] = {0, 3, 5};
  for (int ap = 0; ap < 3; ++ap) {
    Planes A = planes_of(w.U, 4 * n, n2, 3LL * nb, NPLA, w.ld4);
    Planes B = planes_of(w.TT, 4 * n, 4 * n, 1, NPLB, w.ld4);
    cfg.M = (int)n2; cfg.N = (3 - ap) * nv; cfg.K = 4 * nv;
    cfg.a = tc::OpMap{1, nb, 3, ap, 0, (int)n2, w.eU};
    cfg.b = tc::OpMap{1, 1, 0, 0, (ap + 1) * nv, 4 * nv, w.eTT};
    EpiStore<double2> epi;
    epi.out = reinterpret_cast<double2*>(w.V + (long long)slotbase[ap] * n3);
    epi.b_lo = 1; epi.sb_hi = NPAIR * n3; epi.sb_lo = 0;
    epi.sr = 1; epi.cm = ColMap{n2, 0, 0}; epi.N = (3 - ap) * nv;
    DISTIL_TRY((gemm<BF16, NPLA, NPLB>(ctx, "tc_gemm_step_j", A, B, cfg, nb, epi, s)));
  }
  // ---- source: batch (b, c) = nb x 5; X[b][c][pair][k]
  {
    Planes A = planes_of(w.S, n, P2, nb, NPLA, w.ldn);
    Planes B = planes_of(w.Tc, n, n, NSRC, NPLB, w.ldn);
    cfg.M = (int)P2; cfg.N = nv; cfg.K = nv;
    cfg.a = tc::OpMap{NSRC, nb, 1, 0, 0, (int)P2, w.eS};
    cfg.b = tc::OpMap{1, NSRC, 1, 0, 0, nv, w.eTc};
    EpiStore<double2> epi;
    epi.out = reinterpret_cast<double2*>(w.X);
    epi.b_lo = 1; epi.sb_hi = P2 * n; epi.sb_lo = 0;
    epi.sr = n; epi.cm = ColMap{1, 0, 0}; epi.N = nv;
    DISTIL_TRY((gemm<BF16, NPLA, NPLB>(ctx, "tc_gemm_source", A, B, cfg, nb * NSRC, epi, s)));
  }
  // ---- dot
  {
    long long work = P2 * n;
    unsigned gx = (unsigned)((work + 255) / 256);
    if (gx > 1024) gx = 1024;
    Launch L(ctx, "dot", s);
    dot_kernel<double, 16><<<dim3(gx, nb), 256, 0, s>>>(w.V, w.X, nv, nb, Cout, cs_a, cs_b);
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
  MixedWs w = carve_mixed(ar, sch, nv, nb);
  if (!ar.fits()) {
    set_error("correlate: workspace too small");
    return DISTIL_ENOMEM;
  }
  const long long T3 = comb3(nv), n4 = 4LL * nv;
  Cx<double>* Cd = reinterpret_cast<Cx<double>*>(C);
  for (int t = 0; t < nt; ++t) {
    const double* g_snk = prof + (prof_per_t ? (long long)t * nb * nv : 0);
    for (int q = 0; q < np; ++q) {
      const double2* phs = (const double2*)phi_snk + ((long long)t * np + q) * T3;
      const double2* ph0 = (const double2*)phi_src + (long long)q * T3;
      const float2* ta = (const float2*)tau + (long long)t * n4 * n4;
      Cx<double>* Cq = Cd + (long long)q * nb * nb * nt + t;
      const long long ca = (long long)nb * nt, cb = nt;
      int st;
      if (mode == DISTIL_MIXED_FP16X6)
        st = run_tp_mixed<false, true, 3, 4>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, ca, cb, s);
      else if (mode == DISTIL_MIXED_BF16X6)
        st = run_tp_mixed<true, true, 3, 4>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, ca, cb, s);
      else if (mode == DISTIL_MIXED_BF16X3)
        st = run_tp_mixed<true, true, 2, 2>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, ca, cb, s);
      else
        st = run_tp_mixed<false, false, 2, 2>(ctx, sch, phs, ph0, ta, g_snk, prof, nv, nb, w, Cq, ca, cb, s);
      if (st != DISTIL_OK) return st;
    }
  }
  return DISTIL_OK;
}

}  // namespace distil
