// Split-precision complex GEMM on tcgen05 tensor cores.
//
//   D[b](m, n) = sum_k A[b](m, k) * B[b](n, k)          (complex)
//
// A and B arrive pre-split: each complex operand is a stack of 2*NA (2*NB)
// real 16-bit planes (piece p, re/im), K contiguous, read by TMA with the
// swizzle that matches the K chunk (32/64/128-byte rows).  For every K step
// and every product (pa, pb, acc) of the split scheme four MMAs update the
// accumulator pair `acc` in TMEM:
//   D_re[acc] += A_re[pa] B_re[pb] + (-A_im[pa]) B_im[pb]   (negate-A descriptor)
//   D_im[acc] += A_re[pa] B_im[pb] + A_im[pa] B_re[pb]
// Two accumulator pairs exist so that the leading product of a fixed-point
// split (integer-valued slices) sums exactly in its own FP32 accumulator,
// whatever the tensor core's accumulation rounding; every scheme puts at
// least one product into each pair.  The epilogue scales both by
// 2^(eA[row] + eB[col] - shift) (the second also by w1, all exact powers of
// two) and hands the pair to the functor, which keeps D = D[0] + D[1] as a
// double-float.
//
// One CTA computes a 128 x NT tile: warp 0 issues TMA loads into a STAGES-deep
// ring, warp 1 allocates TMEM and issues the MMAs, and 8 epilogue warps (two
// per TMEM lane quarter, each owning half of the columns) read the
// accumulators back (tcgen05.ld) and hand 16-column slices to the epilogue
// functor.  All waits are bounded (tc.cuh).
#pragma once
#include "common.cuh"
#include "tc.cuh"

namespace distil {
namespace tc {

struct OpMap {
  int bdiv, bmod;   // operand batch coordinate = ((batch / bdiv) % bmod) * bmul + badd
  int bmul, badd;
  int row_off;      // added to the tile's first row
  int rows;         // rows per batch coordinate (indexing of the exponent array)
  const int* exps;  // per-row power-of-two exponents [coord][rows] (null: 0)
  __device__ __forceinline__ int coord(int batch) const { return ((batch / bdiv) % bmod) * bmul + badd; }
  __device__ __forceinline__ int exp_of(int c, int r) const { return exps ? exps[(long long)c * rows + r] : 0; }
};

struct GemmCfg {
  int M, N, K;
  OpMap a, b;
  int nprod;
  int pa[6], pb[6], acc[6];
  float w1;   // weight of the second accumulator pair
  int shift;  // D *= 2^(eA + eB - shift)
  unsigned* err;
};

template <int NT, int KC, int NPLA, int NPLB>
struct TileGeom {
  static constexpr int SWZ = KC * 2;  // bytes per tile row
  static constexpr int A_PLANE = 128 * SWZ;
  static constexpr int B_PLANE = NT * SWZ;
  static constexpr int A_STAGE = NPLA * A_PLANE;
  static constexpr int B_STAGE = NPLB * B_PLANE;
  static constexpr int STAGE = A_STAGE + B_STAGE;
};

template <int NT, int KC, int NPLA, int NPLB, int STAGES>
constexpr size_t gemm_smem_bytes() {
  return (size_t)STAGES * TileGeom<NT, KC, NPLA, NPLB>::STAGE + 1024 /*align*/ + 256 /*barriers*/;
}

constexpr int TC_THREADS = 64 + 8 * 32;  // producer, MMA issuer, 8 epilogue warps

template <int NT, int KC, int NPLA, int NPLB, int STAGES, bool BF16, class Epi>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   GemmCfg cfg, Epi epi) {
  using G = TileGeom<NT, KC, NPLA, NPLB>;
  static_assert(NT % 16 == 0 && NT >= 32 && NT <= 128, "N tile");
  static_assert(KC == 16 || KC == 32 || KC == 64, "K chunk");
  // a CTA of a launch that already hit a timeout does nothing; the epilogue
  // may declare a tile empty (no output it keeps) before anything is set up
  if (cfg.err && *(volatile unsigned*)cfg.err) return;
  if (epi.skip_tile(blockIdx.y, blockIdx.x, blockIdx.z)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * G::A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * G::B_STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);
  uint32_t* abort_flag = tslot + 1;
  uint32_t* issued_s = tslot + 2;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tile = blockIdx.x, m_tile = blockIdx.y, batch = blockIdx.z;
  const int nk = (cfg.K + KC - 1) / KC;
  constexpr uint32_t TCOLS = 4 * NT;  // D0_re | D0_im | D1_re | D1_im

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *abort_flag = 0;
    *issued_s = 0;
    fence_mbar_init();
    tma_prefetch(&mapA);
    tma_prefetch(&mapB);
  }
  if (warp == 1) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int ca = cfg.a.coord(batch);
  const int cb = cfg.b.coord(batch);

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&empty[s], ph ^ 1, cfg.err, TC_ERR_EMPTY_WAIT) || *(volatile uint32_t*)abort_flag) {
        *(volatile uint32_t*)abort_flag = 1;
        break;
      }
      mbar_arrive_expect_tx(&full[s], G::STAGE);
      tma_load_4d(&mapA, &full[s], sA + s * G::A_STAGE, kb * KC, m_tile * 128 + cfg.a.row_off, 0, ca);
      tma_load_4d(&mapB, &full[s], sB + s * G::B_STAGE, kb * KC, n_tile * NT + cfg.b.row_off, 0, cb);
      ++issued;
    }
    *(volatile uint32_t*)issued_s = issued;
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    const uint32_t id = idesc_f16(128, NT, BF16, false);
    const uint32_t idn = idesc_f16(128, NT, BF16, true);
    uint32_t started = 0;  // bit a: accumulator pair a has been written
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&full[s], ph, cfg.err, TC_ERR_FULL_WAIT) || *(volatile uint32_t*)abort_flag) {
        *(volatile uint32_t*)abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * G::A_STAGE);
      const uint32_t b0 = smem_u32(sB + s * G::B_STAGE);
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        for (int p = 0; p < cfg.nprod; ++p) {
          const uint32_t ar = a0 + (2 * cfg.pa[p]) * G::A_PLANE + ks * 32;
          const uint32_t ai = ar + G::A_PLANE;
          const uint32_t br = b0 + (2 * cfg.pb[p]) * G::B_PLANE + ks * 32;
          const uint32_t bi = br + G::B_PLANE;
          const uint64_t dar = smem_desc(ar, G::SWZ), dai = smem_desc(ai, G::SWZ);
          const uint64_t dbr = smem_desc(br, G::SWZ), dbi = smem_desc(bi, G::SWZ);
          const int a = cfg.acc[p];
          const uint32_t d = tmem + (uint32_t)(a * 2 * NT);
          const uint32_t accum = (started >> a) & 1u;
          mma_f16(d, dar, dbr, id, accum);
          mma_f16(d, dai, dbi, idn, 1u);
          mma_f16(d + NT, dar, dbi, id, accum);
          mma_f16(d + NT, dai, dbr, id, 1u);
          started |= 1u << a;
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accf);  // fires once every MMA above has completed (also on abort)
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;             // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;   // which half of the NT columns
    bool ok = mbar_wait(accf, 0, cfg.err, TC_ERR_ACC_WAIT);
    ok = __all_sync(0xffffffffu, ok && !*(volatile uint32_t*)abort_flag);  // warp-uniform for tcgen05.ld
    tc_fence_after();
    if (ok) {
      const int row = m_tile * 128 + q * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
      const int ea = (row < cfg.M) ? cfg.a.exp_of(ca, cfg.a.row_off + row) : 0;
#pragma unroll 1
      for (int c = half * (NT / 32); c < (half + 1) * (NT / 32); ++c) {
        uint32_t r0[16], i0[16], r1[16], i1[16];
        tmem_ld16(tl + c * 16, r0);
        tmem_ld16(tl + NT + c * 16, i0);
        tmem_ld16(tl + 2 * NT + c * 16, r1);
        tmem_ld16(tl + 3 * NT + c * 16, i1);
        tmem_wait_ld();
        const int col0 = n_tile * NT + c * 16;
        if (row < cfg.M) {
          float re0[16], re1[16], im0[16], im1[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int col = col0 + e;
            const int eb = (col < cfg.N) ? cfg.b.exp_of(cb, cfg.b.row_off + col) : 0;
            const float f = pow2f(ea + eb - cfg.shift);  // exact power-of-two scalings
            const float f1 = f * cfg.w1;
            re0[e] = __uint_as_float(r0[e]) * f;
            im0[e] = __uint_as_float(i0[e]) * f;
            re1[e] = __uint_as_float(r1[e]) * f1;
            im1[e] = __uint_as_float(i1[e]) * f1;
          }
          epi(batch, row, col0, re0, re1, im0, im1);
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile uint32_t*)abort_flag) {
    // drain: wait (bounded) for the last load of every stage, so no copy
    // lands in shared memory after the CTA has exited
    const int issued = (int)*(volatile uint32_t*)issued_s;
    for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
      if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, cfg.err, TC_ERR_DRAIN)) break;
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

}  // namespace tc
}  // namespace distil
