// Public split-precision complex GEMM (distil_cgemm): C[b] = A[b] B[b]^T for
// complex64 operands, through the same tensor-core engine and split schemes
// as the correlator.  Operands are scaled by powers of two, split into 16-bit
// planes in the workspace, multiplied with FP32 accumulation in TMEM, and
// written back as complex64.
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

using tc::Planes;

// planes [batch][NPL][rows][ld] of s * X, X [batch][rows][K] complex64.
template <bool BF16, int NP>
__global__ void split_rows_kernel(const float2* __restrict__ X, long long rows, long long K, long long batch,
                                  const unsigned* __restrict__ mx, typename tc::Piece<BF16>::T* __restrict__ P,
                                  long long ld) {
  constexpr int NPL = 2 * NP;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= batch * rows * K) return;
  const long long b = e / (rows * K), r = (e / K) % rows, k = e % K;
  const float s = pow2_scale(__uint_as_float(*mx));
  const float2 x = X[e];
  auto* d = P + b * NPL * rows * ld + r * ld + k;
  store_split<BF16, NP>(d, rows * ld, 0, x.x * s);
  store_split<BF16, NP>(d, rows * ld, 1, x.y * s);
}

__global__ void gemm_factor_kernel(const unsigned* mx, float* f) {
  f[0] = 1.f / (pow2_scale(__uint_as_float(mx[0])) * pow2_scale(__uint_as_float(mx[1])));
}

size_t cgemm_workspace(int mode, long long M, long long N, long long K, long long batch) {
  const int NPL = 2 * scheme_of(mode).np;
  Arena ar;
  ar.take<float>(16);
  ar.take<uint16_t>(batch * NPL * M * tc::pad64(K));
  ar.take<uint16_t>(batch * NPL * N * tc::pad64(K));
  return ar.used + 256;
}

template <bool BF16, int NP>
static int cgemm_run(distil_ctx* ctx, const Scheme& sch, const float2* A, const float2* B, float2* C, int M, int N,
                     int K, int batch, void* ws, size_t ws_bytes, cudaStream_t s) {
  using P16 = typename tc::Piece<BF16>::T;
  constexpr int NPL = 2 * NP;
  const long long ld = tc::pad64(K);
  Arena ar(ws, ws_bytes);
  float* sc = ar.take<float>(16);
  P16* PA = ar.take<P16>((long long)batch * NPL * M * ld);
  P16* PB = ar.take<P16>((long long)batch * NPL * N * ld);
  if (!ar.fits()) {
    set_error("distil_cgemm: workspace too small");
    return DISTIL_ENOMEM;
  }
  unsigned* mx = reinterpret_cast<unsigned*>(sc);
  DISTIL_CUDA(cudaMemsetAsync(sc, 0, 16 * sizeof(float), s));
  {
    Launch L(ctx, "cgemm_split", s);
    maxabs_kernel<float><<<128, 256, 0, s>>>((const Cx<float>*)A, (long long)batch * M * K, mx);
    maxabs_kernel<float><<<128, 256, 0, s>>>((const Cx<float>*)B, (long long)batch * N * K, mx + 1);
    gemm_factor_kernel<<<1, 1, 0, s>>>(mx, sc + 2);
    long long ea = (long long)batch * M * K, eb = (long long)batch * N * K;
    split_rows_kernel<BF16, NP><<<(unsigned)((ea + 255) / 256), 256, 0, s>>>(A, M, K, batch, mx, PA, ld);
    split_rows_kernel<BF16, NP><<<(unsigned)((eb + 255) / 256), 256, 0, s>>>(B, N, K, batch, mx + 1, PB, ld);
  }
  DISTIL_LAUNCH_CHECK();
  tc::GemmCfg cfg{};
  cfg.M = M; cfg.N = N; cfg.K = K;
  cfg.a = tc::OpMap{1, batch, 1, 0, 0};
  cfg.b = tc::OpMap{1, batch, 1, 0, 0};
  cfg.nprod = sch.nprod;
  for (int i = 0; i < sch.nprod; ++i) { cfg.pa[i] = sch.pa[i]; cfg.pb[i] = sch.pb[i]; }
  cfg.err = ctx->d_error;
  Planes pa{PA, K, M, NPL, batch, ld, (long long)M * ld, (long long)NPL * M * ld};
  Planes pb{PB, K, N, NPL, batch, ld, (long long)N * ld, (long long)NPL * N * ld};
  EpiC64 epi;
  epi.out = C; epi.b_lo = 1; epi.sb_hi = (long long)M * N; epi.sb_lo = 0; epi.sr = N; epi.N = N;
  epi.factor = sc + 2;
  constexpr int KC = NP == 2 ? 32 : 16;
  if (N > 128)
    return tc::launch_gemm<256, KC, NPL, NP == 2 ? 2 : 3, BF16>(ctx, "tc_gemm_cgemm", pa, pb, cfg, batch, epi, s);
  if (N > 64)
    return tc::launch_gemm<128, KC, NPL, NP == 2 ? 3 : 4, BF16>(ctx, "tc_gemm_cgemm", pa, pb, cfg, batch, epi, s);
  return tc::launch_gemm<64, KC, NPL, NP == 2 ? 3 : 4, BF16>(ctx, "tc_gemm_cgemm", pa, pb, cfg, batch, epi, s);
}

int cgemm_mixed(distil_ctx* ctx, int mode, const void* A, const void* B, void* C, int M, int N, int K, int batch,
                void* ws, size_t ws_bytes, cudaStream_t s) {
  const Scheme sch = scheme_of(mode);
  if (mode == DISTIL_MIXED_BF16X6)
    return cgemm_run<true, 3>(ctx, sch, (const float2*)A, (const float2*)B, (float2*)C, M, N, K, batch, ws, ws_bytes, s);
  if (mode == DISTIL_MIXED_BF16X3)
    return cgemm_run<true, 2>(ctx, sch, (const float2*)A, (const float2*)B, (float2*)C, M, N, K, batch, ws, ws_bytes, s);
  return cgemm_run<false, 2>(ctx, sch, (const float2*)A, (const float2*)B, (float2*)C, M, N, K, batch, ws, ws_bytes, s);
}

}  // namespace distil
