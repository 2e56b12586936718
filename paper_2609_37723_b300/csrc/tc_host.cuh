// Host side of the tensor-core GEMM: launch wrappers of the one-tile,
// persistent and resident-A kernels, with the checks of their operand
// plane images.
#pragma once
#include "common.cuh"
#include "prof.cuh"
#include "tc_gemm.cuh"

namespace distil {
namespace tc {

// Checks of a launch against the plane images it reads: plane counts, K
// blocks, coordinates, first rows on 8-row boundaries, and every tile's rows
// inside the image, so no bulk copy reads outside the buffers.
inline bool images_fit(const char* name, const PlaneImg& A, const PlaneImg& B, const GemmCfg& cfg, int npla,
                       int nplb, int nt, long long m_tiles, long long n_tiles, int batch) {
  const long long kb = (cfg.K + 15) / 16;
  auto coord_max = [batch](const OpMap& m) {
    const long long q = (long long)(batch - 1) / m.bdiv;
    const long long top = (q < m.bmod - 1 ? q : m.bmod - 1);
    return top * m.bmul + m.badd;
  };
  bool ok = A.planes == npla && B.planes == nplb && A.p0 >= 0 && B.p0 >= 0 && A.p0 + A.planes <= A.ptot &&
            B.p0 + B.planes <= B.ptot && kb <= A.kblocks && kb <= B.kblocks;
  ok = ok && cfg.a.bdiv > 0 && cfg.a.bmod > 0 && cfg.b.bdiv > 0 && cfg.b.bmod > 0 && cfg.a.bmul >= 0 &&
       cfg.b.bmul >= 0 && cfg.a.badd >= 0 && cfg.b.badd >= 0;
  ok = ok && coord_max(cfg.a) < A.coords && coord_max(cfg.b) < B.coords;
  ok = ok && cfg.a.row_off >= 0 && cfg.b.row_off >= 0 && cfg.a.row_off % 8 == 0 && cfg.b.row_off % 8 == 0;
  ok = ok && cfg.a.row_off + m_tiles * 128 <= A.rows_pad && cfg.b.row_off + n_tiles * nt <= B.rows_pad;
  ok = ok && cfg.a.row_off + cfg.M <= A.rows && cfg.b.row_off + cfg.N <= B.rows;
  ok = ok && !(reinterpret_cast<uintptr_t>(A.base) & 15) && !(reinterpret_cast<uintptr_t>(B.base) & 15);
  if (!ok)
    set_error("%s: operand images do not cover the launch (M=%d N=%d K=%d batch=%d, planes %d/%d)", name, cfg.M,
              cfg.N, cfg.K, batch, A.planes, B.planes);
  return ok;
}

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
int launch_gemm(distil_ctx* ctx, const char* name, const PlaneImg& A, const PlaneImg& B, const GemmCfg& cfg_in,
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
  constexpr size_t smem = gemm_smem_bytes<NT, KC, NPLA, NPLB, STAGES>();
  static_assert(smem <= 232448, "shared memory");
  auto kern = tc_gemm_kernel<NT, KC, NPLA, NPLB, STAGES, BF16, NACC, Epi>;
  static bool attr = false;
  if (!attr) {
    DISTIL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long n_tiles = (cfg.N + NT - 1) / NT, m_tiles = (cfg.M + 127) / 128;
  if (!images_fit(name, A, B, cfg, NPLA, NPLB, NT, m_tiles, n_tiles, batch)) return DISTIL_EINVAL;
  const long long total = n_tiles * m_tiles * batch;
  if (total > 0x7fffffffLL) {
    set_error("%s: too many tiles", name);
    return DISTIL_EINVAL;
  }
  {
    Launch L(ctx, name, s);
    kern<<<(unsigned)total, TC_THREADS, smem, s>>>(A, B, cfg, epi, (int)n_tiles, (int)m_tiles);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

// Persistent launch: min(tiles, SMs) CTAs walk the 128 x NT tiles with
// NSETS accumulator sets in TMEM.
template <int NT, int KC, int NPLA, int NPLB, int STAGES, bool BF16, int NACC = 2, int NSETS = 2, class Epi>
int launch_gemm_persistent(distil_ctx* ctx, const char* name, const PlaneImg& A, const PlaneImg& B,
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
  constexpr size_t smem = gemm_smem_bytes<NT, KC, NPLA, NPLB, STAGES>();
  static_assert(smem <= 232448, "shared memory");
  auto kern = tc_gemm_persistent_kernel<NT, KC, NPLA, NPLB, STAGES, BF16, NACC, Epi, NSETS>;
  static bool attr = false;
  if (!attr) {
    DISTIL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long n_tiles = (cfg.N + NT - 1) / NT, m_tiles = (cfg.M + 127) / 128;
  if (!images_fit(name, A, B, cfg, NPLA, NPLB, NT, m_tiles, n_tiles, batch)) return DISTIL_EINVAL;
  const long long total = n_tiles * m_tiles * batch;
  if (total > 0x7fffffffLL) {
    set_error("%s: too many tiles", name);
    return DISTIL_EINVAL;
  }
  const int grid = (int)(total < ctx->sm_count ? total : ctx->sm_count);
  {
    Launch L(ctx, name, s);
    kern<<<grid, TC_THREADS, smem, s>>>(A, B, cfg, epi, (int)n_tiles, (int)m_tiles, (int)total);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

// A-resident persistent launch: K <= NKA * KC; min(tiles, SMs) CTAs, each a
// contiguous range of tiles.
template <int NT, int KC, int NPLA, int NPLB, int NKA, bool BF16, int NACC = 2, class Epi>
int launch_gemm_ares(distil_ctx* ctx, const char* name, const PlaneImg& A, const PlaneImg& B, const GemmCfg& cfg_in,
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
  constexpr size_t smem = (size_t)NKA * G::A_STAGE + (size_t)STAGES * G::B_STAGE + 1024 + 256;
  static_assert(smem <= 232448, "shared memory");
  auto kern = tc_gemm_ares_kernel<NT, KC, NPLA, NPLB, NKA, STAGES, BF16, NACC, Epi>;
  static bool attr = false;
  if (!attr) {
    DISTIL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long long n_tiles = (cfg.N + NT - 1) / NT, m_tiles = (cfg.M + 127) / 128;
  if (!images_fit(name, A, B, cfg, NPLA, NPLB, NT, m_tiles, n_tiles, batch)) return DISTIL_EINVAL;
  const long long total = n_tiles * m_tiles * batch;
  if (total > 0x7fffffffLL) {
    set_error("%s: too many tiles", name);
    return DISTIL_EINVAL;
  }
  const int grid = (int)(total < ctx->sm_count ? total : ctx->sm_count);
  {
    Launch L(ctx, name, s);
    kern<<<grid, TC_THREADS, smem, s>>>(A, B, cfg, epi, (int)n_tiles, (int)m_tiles, (int)total);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

}  // namespace tc
}  // namespace distil
