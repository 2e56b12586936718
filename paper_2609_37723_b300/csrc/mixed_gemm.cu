// Public split-precision complex GEMM (distil_cgemm): C[b] = A[b] B[b]^T for
// complex64 operands, through the same tensor-core engine and split schemes
// as the correlator: rows split into 16-bit pieces with per-row
// power-of-two exponents, products accumulated in TMEM, complex64 out.
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

namespace {
struct BatchRows {  // row r of [batch][rows][K], exact in double-float
  const float2* x;
  long long K;
  __device__ __forceinline__ CDF operator()(long long r, int k) const {
    const float2 v = x[r * K + k];
    return cdf_make(df_make(v.x, 0.f), df_make(v.y, 0.f));
  }
  __device__ __forceinline__ float2 approx(long long r, int k) const { return x[r * K + k]; }
};
}  // namespace

size_t cgemm_workspace(int mode, long long M, long long N, long long K, long long batch) {
  const Scheme sc = scheme_of(mode);
  Arena ar;
  ar.take<int>(batch * (M + N));
  ar.take<uint16_t>(tc::plane_img_elems(K, M, batch, 2 * sc.na));
  ar.take<uint16_t>(tc::plane_img_elems(K, N, batch, 2 * sc.nb));
  return ar.used + 256;
}

template <bool BF16, bool FIXED, int NA, int NB>
static int cgemm_run(distil_ctx* ctx, const Scheme& sch, const float2* A, const float2* B, float2* C, int M, int N,
                     int K, int batch, void* ws, size_t ws_bytes, cudaStream_t s) {
  constexpr int NPLA = 2 * NA, NPLB = 2 * NB;
  Arena ar(ws, ws_bytes);
  int* eA = ar.take<int>((long long)batch * M);
  int* eB = ar.take<int>((long long)batch * N);
  const tc::PlaneImg pa = tc::plane_img(ar.take<uint16_t>(tc::plane_img_elems(K, M, batch, NPLA)), K, M, batch, NPLA);
  const tc::PlaneImg pb = tc::plane_img(ar.take<uint16_t>(tc::plane_img_elems(K, N, batch, NPLB)), K, N, batch, NPLB);
  if (!ar.fits()) {
    set_error("distil_cgemm: workspace too small");
    return DISTIL_ENOMEM;
  }
  // fixed-point FP16: a narrower leading slice for long K keeps the exact
  // hi*hi sums below 2^24 (they grow like 2^2H sqrt(K) for rows of random sign)
  const int H = (FIXED && !BF16) ? (K <= 1024 ? sch.H : K <= 4096 ? 9 : K <= 16384 ? 8 : 7) : sch.H;
  DISTIL_TRY((split_rows<BF16, FIXED, NA>(ctx, "split_cgemm", BatchRows{A, K}, (long long)batch * M, pa, H, eA, s)));
  DISTIL_TRY((split_rows<BF16, FIXED, NB>(ctx, "split_cgemm", BatchRows{B, K}, (long long)batch * N, pb, H, eB, s)));
  tc::GemmCfg cfg{};
  fill_products(cfg, sch);
  cfg.shift = 2 * H;
  cfg.M = M; cfg.N = N; cfg.K = K;
  cfg.a = tc::OpMap{1, batch, 1, 0, 0, M, eA};
  cfg.b = tc::OpMap{1, batch, 1, 0, 0, N, eB};
  cfg.err = ctx->d_error;
  EpiStoreC64 epi{{}, C, (long long)M * N, N, N};
  // the 6-product schemes accumulate in three pairs (exact cross terms)
  constexpr int NACC = NPLA == 6 ? 3 : 2;
  constexpr int NTW = NACC == 3 ? 80 : 128;
  if (N > 64)
    return tc::launch_gemm<NTW, 16, NPLA, NPLB, tc::max_stages<NTW, 16, NPLA, NPLB>(), BF16, NACC>(
        ctx, "tc_gemm_cgemm", pa, pb, cfg, batch, epi, s);
  if (N > 32)
    return tc::launch_gemm<64, 16, NPLA, NPLB, tc::max_stages<64, 16, NPLA, NPLB>(), BF16, NACC>(
        ctx, "tc_gemm_cgemm", pa, pb, cfg, batch, epi, s);
  return tc::launch_gemm<32, 16, NPLA, NPLB, tc::max_stages<32, 16, NPLA, NPLB>(), BF16, NACC>(
      ctx, "tc_gemm_cgemm", pa, pb, cfg, batch, epi, s);
}

int cgemm_mixed(distil_ctx* ctx, int mode, const void* A, const void* B, void* C, int M, int N, int K, int batch,
                void* ws, size_t ws_bytes, cudaStream_t s) {
  const Scheme sch = scheme_of(mode);
  const float2 *a = (const float2*)A, *b = (const float2*)B;
  float2* c = (float2*)C;
  if (mode == DISTIL_MIXED_FP16X6)
    return cgemm_run<false, true, 3, 4>(ctx, sch, a, b, c, M, N, K, batch, ws, ws_bytes, s);
  if (mode == DISTIL_MIXED_BF16X6)
    return cgemm_run<true, true, 3, 4>(ctx, sch, a, b, c, M, N, K, batch, ws, ws_bytes, s);
  if (mode == DISTIL_MIXED_BF16X3)
    return cgemm_run<true, true, 2, 2>(ctx, sch, a, b, c, M, N, K, batch, ws, ws_bytes, s);
  return cgemm_run<false, false, 2, 2>(ctx, sch, a, b, c, M, N, K, batch, ws, ws_bytes, s);
}

}  // namespace distil
