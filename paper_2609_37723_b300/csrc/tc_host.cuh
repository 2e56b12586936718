// Host side of the tensor-core GEMM: TMA tensor maps for stacks of 16-bit
// planes and the launch wrapper of tc_gemm_kernel.
#pragma once
#include <cuda.h>

#include "common.cuh"
#include "prof.cuh"
#include "tc_gemm.cuh"

namespace distil {
namespace tc {

// A stack of 16-bit planes: element (k, row, plane, batch) at
// base + batch*batch_stride + plane*plane_stride + row*ld + k  (elements).
struct Planes {
  void* base;
  long long K, rows, planes, batch;
  long long ld, plane_stride, batch_stride;
};

inline long long pad64(long long k) { return (k + 63) / 64 * 64; }

int encode_planes(CUtensorMap* map, const Planes& t, int box_rows, int kc, bool bf16);

// The kernel's MMA schedule is compiled for the scheme of its plane counts
// and accumulator pairs: the caller's products must be the scheme's; the
// accumulator of each product is the kernel's (written into cfg).
template <int NPLA, int NPLB, int NACC>
bool products_match(GemmCfg& cfg) {
  using P = SchemeProducts<NPLA, NPLB, NACC>;
  bool same = cfg.nprod == P::n;
  for (int p = 0; same && p < P::n; ++p) same = cfg.pa[p] == P::pa[p] && cfg.pb[p] == P::pb[p];
  for (int p = 0; same && p < P::n; ++p) cfg.acc[p] = P::acc[p];
  return same;
}

template <int NT, int KC, int NPLA, int NPLB, int STAGES, bool BF16, int NACC = 2, class Epi>
int launch_gemm(distil_ctx* ctx, const char* name, const Planes& A, const Planes& B, const GemmCfg& cfg_in,
                int batch, const Epi& epi, cudaStream_t s) {
  GemmCfg cfg = cfg_in;
  cfg.wait = (ctx && ctx->wait_limit > 0) ? ctx->wait_limit : TC_WAIT_CYCLES;
  if (cfg.M <= 0 || cfg.N <= 0 || batch <= 0) return DISTIL_OK;
  if (cfg.K <= 0) {
    set_error("%s: K must be positive", name);
    return DISTIL_EINVAL;
  }
  if (!products_match<NPLA, NPLB, NACC>(cfg)) {
    set_error("%s: split products do not match the %dx%d-plane kernel", name, NPLA, NPLB);
    return DISTIL_EINVAL;
  }
  CUtensorMap ma, mb;
  DISTIL_TRY(encode_planes(&ma, A, 128, KC, BF16));
  DISTIL_TRY(encode_planes(&mb, B, NT, KC, BF16));
  constexpr size_t smem = gemm_smem_bytes<NT, KC, NPLA, NPLB, STAGES>();
  static_assert(smem <= 232448, "shared memory");
  auto kern = tc_gemm_kernel<NT, KC, NPLA, NPLB, STAGES, BF16, NACC, Epi>;
  static bool attr = false;
  if (!attr) {
    DISTIL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long n_tiles = (cfg.N + NT - 1) / NT, m_tiles = (cfg.M + 127) / 128;
  const long long total = n_tiles * m_tiles * batch;
  if (total > 0x7fffffffLL) {
    set_error("%s: too many tiles", name);
    return DISTIL_EINVAL;
  }
  {
    Launch L(ctx, name, s);
    kern<<<(unsigned)total, TC_THREADS, smem, s>>>(ma, mb, cfg, epi, (int)n_tiles, (int)m_tiles);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

// Persistent launch: min(tiles, SMs) CTAs walk the 128 x NT tiles.
template <int NT, int KC, int NPLA, int NPLB, int STAGES, bool BF16, int NACC = 2, class Epi>
int launch_gemm_persistent(distil_ctx* ctx, const char* name, const Planes& A, const Planes& B,
                           const GemmCfg& cfg_in, int batch, const Epi& epi, cudaStream_t s) {
  GemmCfg cfg = cfg_in;
  cfg.wait = (ctx && ctx->wait_limit > 0) ? ctx->wait_limit : TC_WAIT_CYCLES;
  if (cfg.M <= 0 || cfg.N <= 0 || batch <= 0) return DISTIL_OK;
  if (cfg.K <= 0) {
    set_error("%s: K must be positive", name);
    return DISTIL_EINVAL;
  }
  if (!products_match<NPLA, NPLB, NACC>(cfg)) {
    set_error("%s: split products do not match the %dx%d-plane kernel", name, NPLA, NPLB);
    return DISTIL_EINVAL;
  }
  CUtensorMap ma, mb;
  DISTIL_TRY(encode_planes(&ma, A, 128, KC, BF16));
  DISTIL_TRY(encode_planes(&mb, B, NT, KC, BF16));
  constexpr size_t smem = gemm_smem_bytes<NT, KC, NPLA, NPLB, STAGES>();
  static_assert(smem <= 232448, "shared memory");
  auto kern = tc_gemm_persistent_kernel<NT, KC, NPLA, NPLB, STAGES, BF16, NACC, Epi>;
  static bool attr = false;
  if (!attr) {
    DISTIL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long n_tiles = (cfg.N + NT - 1) / NT, m_tiles = (cfg.M + 127) / 128;
  const long long total = n_tiles * m_tiles * batch;
  if (total > 0x7fffffffLL) {
    set_error("%s: too many tiles", name);
    return DISTIL_EINVAL;
  }
  const int grid = (int)(total < ctx->sm_count ? total : ctx->sm_count);
  {
    Launch L(ctx, name, s);
    kern<<<grid, TC_THREADS, smem, s>>>(ma, mb, cfg, epi, (int)n_tiles, (int)m_tiles, (int)total);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

// A-resident persistent launch: K <= NKA * KC; min(tiles, SMs) CTAs, each a
// contiguous range of tiles.
template <int NT, int KC, int NPLA, int NPLB, int NKA, bool BF16, int NACC = 2, class Epi>
int launch_gemm_ares(distil_ctx* ctx, const char* name, const Planes& A, const Planes& B, const GemmCfg& cfg_in,
                     int batch, const Epi& epi, cudaStream_t s) {
  GemmCfg cfg = cfg_in;
  cfg.wait = (ctx && ctx->wait_limit > 0) ? ctx->wait_limit : TC_WAIT_CYCLES;
  using G = TileGeom<NT, KC, NPLA, NPLB>;
  constexpr size_t room = 232448 - 1024 - 256 - (size_t)NKA * G::A_STAGE;
  constexpr int ST0 = (int)(room / G::B_STAGE);
  constexpr int STAGES = ST0 > 6 ? 6 : ST0;
  static_assert(STAGES >= 2, "resident A leaves room for a two-stage B ring");
  if (cfg.M <= 0 || cfg.N <= 0 || batch <= 0) return DISTIL_OK;
  if (cfg.K <= 0 || cfg.K > NKA * KC) {
    set_error("%s: K=%d outside (0, %d] of the resident-A kernel", name, cfg.K, NKA * KC);
    return DISTIL_EINVAL;
  }
  if (!products_match<NPLA, NPLB, NACC>(cfg)) {
    set_error("%s: split products do not match the %dx%d-plane kernel", name, NPLA, NPLB);
    return DISTIL_EINVAL;
  }
  CUtensorMap ma, mb;
  DISTIL_TRY(encode_planes(&ma, A, 128, KC, BF16));
  DISTIL_TRY(encode_planes(&mb, B, NT, KC, BF16));
  constexpr size_t smem = (size_t)NKA * G::A_STAGE + (size_t)STAGES * G::B_STAGE + 1024 + 256;
  static_assert(smem <= 232448, "shared memory");
  auto kern = tc_gemm_ares_kernel<NT, KC, NPLA, NPLB, NKA, STAGES, BF16, NACC, Epi>;
  static bool attr = false;
  if (!attr) {
    DISTIL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long n_tiles = (cfg.N + NT - 1) / NT, m_tiles = (cfg.M + 127) / 128;
  const long long total = n_tiles * m_tiles * batch;
  if (total > 0x7fffffffLL) {
    set_error("%s: too many tiles", name);
    return DISTIL_EINVAL;
  }
  const int grid = (int)(total < ctx->sm_count ? total : ctx->sm_count);
  {
    Launch L(ctx, name, s);
    kern<<<grid, TC_THREADS, smem, s>>>(ma, mb, cfg, epi, (int)n_tiles, (int)m_tiles, (int)total);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

}  // namespace tc
}  // namespace distil
