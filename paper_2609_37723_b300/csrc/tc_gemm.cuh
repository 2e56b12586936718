// Split-precision complex GEMM on tcgen05 tensor cores.
//
//   D[b](m, n) = sum_k A[b](m, k) * B[b](n, k)          (complex)
//
// A and B arrive pre-split: each complex operand is a stack of 2*NA (2*NB)
// real 16-bit planes (piece p, re/im) stored as plane images (PlaneImg: the
// shared-memory tile image itself, K in blocks of 16), so every stage
// arrives through plain bulk copies of whole rows of 32 bytes.  For every K step
// and every product (pa, pb, acc) of the split scheme four MMAs update the
// accumulator pair `acc` in TMEM:
//   D_re[acc] += A_re[pa] B_re[pb] + (-A_im[pa]) B_im[pb]   (negate-A descriptor)
//   D_im[acc] += A_re[pa] B_im[pb] + A_im[pa] B_re[pb]
// Two or three accumulator pairs exist (SchemeProducts) so that the products
// of integer slices of a fixed-point split sum exactly in FP32 accumulators
// of their own, whatever the tensor core's accumulation rounding; every
// scheme puts at least one product into each pair.  The epilogue scales
// them by 2^(eA[row] + eB[col] - shift) (the cross-term pairs also by w1,
// all exact powers of two) and hands the leading and the cross-term sums to
// the functor, which keeps D = D[0] + D[1] as a double-float.
//
// One CTA computes a 128 x NT tile: warp 0 issues the bulk copies of a
// STAGES-deep ring, warp 1 allocates TMEM and issues the MMAs, and 8 epilogue warps (two
// per TMEM lane quarter, taking alternate 16-column slices) read the
// accumulators back (tcgen05.ld) and hand 16-column slices to the epilogue
// functor.  All waits are bounded (tc.cuh).
#pragma once
#include "common.cuh"
#include "tc.cuh"

namespace distil {
namespace tc {

// A stack of 16-bit planes in shared-memory tile-image order.  For
// coordinate c, K block kb (elements 16 kb .. 16 kb + 15), plane p and row r
// the 16 elements take 32 contiguous bytes at byte offset
//   ((((c * kblocks + kb) * planes + p) * rows_pad + r) * 32
// with their two 16-byte halves swapped where bit 2 of r is set: the
// 32-byte-swizzled K-major layout the MMA descriptors describe, so the rows
// r0 .. r0 + R - 1 of one (c, kb, p) (r0 a multiple of 8) are one
// contiguous run that a single bulk copy puts in place.  Whole cache lines
// move, where a tensor-map load of 32-byte box rows issued one L2 request
// per 32-byte sector (the L2 tag rate bounded the contractions).  rows_pad
// is rows rounded up to 8 plus 128, so any tile starting below `rows` can
// be copied whole; rows past `rows` only reach outputs that are not kept.
// Elements of the last K block past K must be zero (the writers store them).
// An image stores ptot planes per (c, kb); a GEMM reads `planes` of them
// from plane p0 on (plane_view: a subset of the pieces).
struct PlaneImg {
  void* base;
  long long rows, rows_pad;
  int K, kblocks, planes, coords, ptot, p0;
  // first row of block (c, kb, p), in rows (p counted from p0)
  __host__ __device__ __forceinline__ long long block(long long c, int kb, int p) const {
    return ((c * kblocks + kb) * ptot + p0 + p) * rows_pad;
  }
  // element index of (c, p, r, k)
  __host__ __device__ __forceinline__ long long index(long long c, int p, long long r, int k) const {
    return ((block(c, k >> 4, p) + r) << 4) + ((((k >> 3) ^ (int)(r >> 2)) & 1) << 3) + (k & 7);
  }
  __device__ __forceinline__ const uint8_t* rows_at(long long c, int kb, int p, long long r) const {
    return reinterpret_cast<const uint8_t*>(base) + ((block(c, kb, p) + r) << 5);
  }
};
inline long long img_rows_pad(long long rows) { return (rows + 7) / 8 * 8 + 128; }
inline PlaneImg plane_img(void* base, long long K, long long rows, long long coords, int planes) {
  PlaneImg g;
  g.base = base;
  g.rows = rows;
  g.rows_pad = img_rows_pad(rows);
  g.K = (int)K;
  g.kblocks = (int)((K + 15) / 16);
  g.planes = planes;
  g.coords = (int)coords;
  g.ptot = planes;
  g.p0 = 0;
  return g;
}
// The same image read as its planes p0 .. p0 + np - 1.
inline PlaneImg plane_view(const PlaneImg& g, int p0, int np) {
  PlaneImg v = g;
  v.p0 = g.p0 + p0;
  v.planes = np;
  return v;
}
// 16-bit elements of a plane image
inline long long plane_img_elems(long long K, long long rows, long long coords, int planes) {
  return coords * ((K + 15) / 16) * planes * img_rows_pad(rows) * 16;
}

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
  int pa[8], pb[8], acc[8];
  float w1;   // weight of the cross-term accumulator pairs
  int shift;  // D *= 2^(eA + eB - shift)
  unsigned* err;
  long long wait;  // limit of the pipeline waits in clock cycles (teardown waits keep TC_WAIT_CYCLES)
  int order;       // tile order of the persistent and one-tile kernels (tile_at)
};

// Output tile of linear tile index t.  order 0: n fastest, then m, then
// batch.  order 1 (B reuse): m fastest, then the b.bdiv consecutive batches
// that share one B operand, then n, then the rest of the batch -- the tiles
// that read the same B tile run back to back, so it is fetched from HBM
// once and served from L2 to the others (step i: 2 x 12 uses per B tile).
struct TileIdx {
  int n_tile, m_tile, batch;
};
__device__ __forceinline__ TileIdx tile_at(int t, int n_tiles, int m_tiles, const GemmCfg& cfg) {
  TileIdx r;
  if (cfg.order == 1) {
    const int br = cfg.b.bdiv;
    r.m_tile = t % m_tiles;
    const int q = t / m_tiles;
    const int bi = q % br, q2 = q / br;
    r.n_tile = q2 % n_tiles;
    r.batch = (q2 / n_tiles) * br + bi;
  } else {
    r.n_tile = t % n_tiles;
    const int rest = t / n_tiles;
    r.m_tile = rest % m_tiles;
    r.batch = rest / m_tiles;
  }
  return r;
}

// Products of the split schemes, by operand planes: 3 x 4 pieces (6
// products, fixed point) or 2 x 2 pieces (3 products).  A product (pa, pb,
// acc) adds A[pa] B[pb] into accumulator pair acc.  The 6-product scheme
// comes with two or three accumulator pairs (NACC):
//   NACC = 2: hi*hi | every cross term
//   NACC = 3: hi*hi | hi*mid + mid*hi | the second-order terms
// With three pairs the first two hold sums of products of integer slices
// only, which the FP32 accumulation adds exactly while the partial sums stay
// below 2^24; the third holds the pre-scaled second-order terms, about 2^-11
// of the second, whose inexact accumulation no longer drifts with K at the
// level of the result.  The 3-product schemes have two pairs.
template <int NPLA, int NPLB, int NACC>
struct SchemeProducts;
template <>
struct SchemeProducts<6, 8, 2> {
  static constexpr int n = 6;
  static constexpr int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 3, 2, 0}, acc[6] = {0, 1, 1, 1, 1, 1};
};
template <>
struct SchemeProducts<6, 8, 3> {
  static constexpr int n = 6;
  static constexpr int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 3, 2, 0}, acc[6] = {0, 1, 1, 2, 2, 2};
};
// 4 x 4 pieces (hi, mid, mid 2^-W, lo 2^-W on both sides), 8 products: the
// six of the 3 x 4 scheme plus the third-order lo*mid and mid*lo, which the
// 6-product scheme drops (a term of relative size 2^-(W+2+2H) per product
// that does not shrink with the leading-slice width H).  Three pairs:
// hi*hi | hi*mid + mid*hi | the second- and third-order terms.
template <>
struct SchemeProducts<8, 8, 3> {
  static constexpr int n = 8;
  static constexpr int pa[8] = {0, 0, 1, 0, 3, 1, 3, 2}, pb[8] = {0, 1, 0, 3, 0, 2, 2, 3},
                       acc[8] = {0, 1, 1, 2, 2, 2, 2, 2};
};
// The second-order class alone (one accumulator pair), for a second pass
// over the same operands after <4, 4, 2> has accumulated hi*hi | hi*mid +
// mid*hi from the leading two pieces of each side: 3 x 4 pieces (the
// <6, 8, 3> products of pair 2) and 4 x 4 pieces (those of <8, 8, 3>).
template <>
struct SchemeProducts<6, 8, 1> {
  static constexpr int n = 3;
  static constexpr int pa[3] = {0, 1, 2}, pb[3] = {3, 2, 0}, acc[3] = {0, 0, 0};
};
// the same, with the B operand viewed as the pieces [mid', lo, hi] (the
// first six planes of a B image stored in the piece order mid', lo, hi, mid,
// whose last four planes are the [hi, mid] of the first pass)
template <>
struct SchemeProducts<6, 6, 1> {
  static constexpr int n = 3;
  static constexpr int pa[3] = {0, 1, 2}, pb[3] = {1, 0, 2}, acc[3] = {0, 0, 0};
};
template <>
struct SchemeProducts<8, 8, 1> {
  static constexpr int n = 5;
  static constexpr int pa[5] = {0, 3, 1, 3, 2}, pb[5] = {3, 0, 2, 2, 3}, acc[5] = {0, 0, 0, 0, 0};
};
template <>
struct SchemeProducts<4, 4, 2> {
  static constexpr int n = 3;
  static constexpr int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0}, acc[3] = {0, 1, 1};
};

// TMEM columns an allocation of `cols` needs: a power of two >= 32.
__host__ __device__ constexpr uint32_t tmem_alloc_cols(uint32_t cols) {
  uint32_t a = 32;
  while (a < cols) a <<= 1;
  return a;
}

// One real MMA: A plane, B plane, accumulator (pair * 2 + re/im), negate B,
// first write of its accumulator.
struct MmaOp {
  int ap, bp, dsel, negb, first;
};

// The 4 * nprod real MMAs of a 16-deep K step, grouped by A plane:
//   A_re[pa]: D_re += A_re B_re[pb],   D_im += A_re B_im[pb]
//   A_im[pa]: D_re += A_im (-B_im[pb]) (negate-B descriptor),  D_im += A_im B_re[pb]
// Built at compile time, so the single issuing thread only adds constant
// offsets to two descriptors per stage and keeps the tensor pipe fed (a
// schedule decoded at run time left it waiting on the issuer).
template <int NPLA, int NPLB, int NACC>
struct MmaSchedule {
  using P = SchemeProducts<NPLA, NPLB, NACC>;
  static constexpr int n = 4 * P::n;
  MmaOp ops[4 * P::n];
  constexpr MmaSchedule() : ops{} {
    int k = 0;
    bool written[6] = {false, false, false, false, false, false};
    for (int pa = 0; pa < NPLA / 2; ++pa) {
      for (int part = 0; part < 2; ++part) {
        for (int p = 0; p < P::n; ++p) {
          if (P::pa[p] != pa) continue;
          const int br = 2 * P::pb[p], bi = br + 1, d = 2 * P::acc[p];
          // D_re first, then D_im
          const int b0 = part ? bi : br, b1 = part ? br : bi;
          ops[k] = MmaOp{2 * pa + part, b0, d, part, written[d] ? 0 : 1};
          written[d] = true;
          ++k;
          ops[k] = MmaOp{2 * pa + part, b1, d + 1, 0, written[d + 1] ? 0 : 1};
          written[d + 1] = true;
          ++k;
        }
      }
    }
  }
};

// Epilogue functors see each 16-column slice of a row, with a per-thread
// State that lives across the slices of a tile: begin() before the first,
// end() after the last (called by all 32 lanes of the warp together, also
// for rows past M, so it may use warp shuffles).  Stateless epilogues
// derive from this.
struct EpiStateless {
  struct State {};
  // before the accumulator is waited for: loads the tile's slices will use
  // (row, first column of the warp's first slice)
  __device__ __forceinline__ void prefetch(State&, int, int, int) const {}
  __device__ __forceinline__ void begin(State&) const {}
  __device__ __forceinline__ void end(State&, int) const {}
};

template <int NT, int KC, int NPLA, int NPLB>
struct TileGeom {
  static_assert(KC == 16, "plane images hold K in blocks of 16");
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
static_assert(2 * 8 * 6 + 5 * 8 + 16 <= 256, "barrier area: 2 x 6 ring barriers, 5 others, 3 words");

// Deepest ring (at most 6 stages) that fits the 227 KB of shared memory.
template <int NT, int KC, int NPLA, int NPLB>
constexpr int max_stages() {
  constexpr size_t room = 232448 - 1024 - 256;
  constexpr int s = (int)(room / TileGeom<NT, KC, NPLA, NPLB>::STAGE);
  return s > 6 ? 6 : s;
}

constexpr int TC_THREADS = 64 + 8 * 32;  // producer, MMA issuer, 8 epilogue warps

// The NPL planes of K block kb, rows r0 .. r0 + R - 1 of coordinate c, into
// consecutive R x 32-byte plane tiles at dst: one bulk copy per plane.
template <int NPL, int R>
__device__ __forceinline__ void load_planes(const PlaneImg& g, uint8_t* dst, uint64_t* bar, int kb, int c, int r0) {
#pragma unroll
  for (int p = 0; p < NPL; ++p) bulk_load(dst + p * (R * 32), g.rows_at(c, kb, p, r0), R * 32, bar);
}
template <int NT, int KC, int NPLA, int NPLB>
__device__ __forceinline__ void load_stage(const PlaneImg& ga, const PlaneImg& gb, uint8_t* sa, uint8_t* sb,
                                           uint64_t* bar, int kb, int ca, int ra, int cb, int rb) {
  load_planes<NPLA, 128>(ga, sa, bar, kb, ca, ra);
  load_planes<NPLB, NT>(gb, sb, bar, kb, cb, rb);
}

// Exponents of the output tile's row and columns for one epilogue warp,
// loaded before the accumulator is waited for: ea of the thread's row, and
// those of the (at most 64) columns of the warp's slices c = half, half + 2,
// ... packed two per lane: ebp[r] of lane l is column slot 32 r + l, slot
// 16 s + e being element e of the warp's s-th slice.
template <int NT>
__device__ __forceinline__ void tile_exps(const GemmCfg& cfg, int ca, int cb, int row, int n_tile, int half, int lane,
                                          int& ea, int (&ebp)[2]) {
  static_assert(NT <= 128, "two column slots per lane");
  ea = (row < cfg.M) ? cfg.a.exp_of(ca, cfg.a.row_off + row) : 0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int slot = 32 * r + lane, c = half + 2 * (slot >> 4);
    const int col = n_tile * NT + c * 16 + (slot & 15);
    ebp[r] = (c < NT / 16 && col < cfg.N) ? cfg.b.exp_of(cb, cfg.b.row_off + col) : 0;
  }
}

// Epilogue of one 16-column slice c of a tile for this thread's row: read
// the NACC accumulator pairs at TMEM address tl (D0_re | D0_im | D1_re |
// D1_im [| D2_re | D2_im], NT columns each; every lane of the warp takes
// part), scale by the exact powers of two 2^(eA + eB - shift) (and w1 for
// the cross terms, D1 + D2 summed in FP32) and hand the pair to the
// epilogue functor.  ea, ebp: tile_exps of this warp (slice c is the
// warp's slice (c - half) / 2).
template <int NT, int NACC, class Epi>
__device__ __forceinline__ void epi_slice(const Epi& epi, typename Epi::State& st, const GemmCfg& cfg, uint32_t tl,
                                          int c, int half, int batch, int row, int n_tile, int ea,
                                          const int (&ebp)[2]) {
  uint32_t r0[16], i0[16], r1[16], i1[16], r2[16], i2[16];
  tmem_ld16(tl + c * 16, r0);
  tmem_ld16(tl + NT + c * 16, i0);
  if constexpr (NACC >= 2) {
    tmem_ld16(tl + 2 * NT + c * 16, r1);
    tmem_ld16(tl + 3 * NT + c * 16, i1);
  }
  if constexpr (NACC == 3) {
    tmem_ld16(tl + 4 * NT + c * 16, r2);
    tmem_ld16(tl + 5 * NT + c * 16, i2);
  }
  tmem_wait_ld();
  const int col0 = n_tile * NT + c * 16;
  const int sl = (c - half) >> 1;                  // the warp's slice index
  const int ebs = (sl >> 1) ? ebp[1] : ebp[0];     // lane register holding its slots
  int eb[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) eb[e] = __shfl_sync(0xffffffffu, ebs, ((sl & 1) << 4) + e);
  if (row < cfg.M) {
    float re0[16], re1[16], im0[16], im1[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float f = pow2f(ea + eb[e] - cfg.shift);  // exact power-of-two scalings
      const float f1 = f * cfg.w1;
      if constexpr (NACC == 1) {
        // a pass of cross terms only: its one pair carries the w1 weight
        re0[e] = 0.f;
        im0[e] = 0.f;
        re1[e] = __uint_as_float(r0[e]) * f1;
        im1[e] = __uint_as_float(i0[e]) * f1;
      } else {
        float x1 = __uint_as_float(r1[e]), y1 = __uint_as_float(i1[e]);
        if constexpr (NACC == 3) {
          x1 += __uint_as_float(r2[e]);
          y1 += __uint_as_float(i2[e]);
        }
        re0[e] = __uint_as_float(r0[e]) * f;
        im0[e] = __uint_as_float(i0[e]) * f;
        re1[e] = x1 * f1;
        im1[e] = y1 * f1;
      }
    }
    epi(st, batch, row, col0, re0, re1, im0, im1);
  }
}

template <int NT, int KC, int NPLA, int NPLB, int STAGES, bool BF16, int NACC, class Epi>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(PlaneImg ga, PlaneImg gb, GemmCfg cfg, Epi epi, int n_tiles, int m_tiles) {
  using G = TileGeom<NT, KC, NPLA, NPLB>;
  static_assert(NT % 16 == 0 && NT >= 32 && NT <= 128 && 2 * NACC * NT <= 512, "N tile / TMEM columns");
  // a CTA of a launch that already hit a timeout does nothing; the epilogue
  // may declare a tile empty (no output it keeps) before anything is set up
  if (cfg.err && *(volatile unsigned*)cfg.err) return;
  const TileIdx ti = tile_at((int)blockIdx.x, n_tiles, m_tiles, cfg);
  if (epi.skip_tile(ti.m_tile, ti.n_tile, ti.batch)) return;
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
  const int n_tile = ti.n_tile, m_tile = ti.m_tile, batch = ti.batch;
  const int nk = (cfg.K + KC - 1) / KC;
  constexpr uint32_t TCOLS = tmem_alloc_cols(2 * NACC * NT);  // D0_re | D0_im | D1_re | D1_im [| D2_re | D2_im]

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *abort_flag = 0;
    *issued_s = 0;
    fence_mbar_init();
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
    // ---------------------------------------------------------------- copy producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&empty[s], ph ^ 1, cfg.err, TC_ERR_EMPTY_WAIT, cfg.wait) || *(volatile uint32_t*)abort_flag) {
        *(volatile uint32_t*)abort_flag = 1;
        break;
      }
      mbar_arrive_expect_tx(&full[s], G::STAGE);
      load_stage<NT, KC, NPLA, NPLB>(ga, gb, sA + s * G::A_STAGE, sB + s * G::B_STAGE, &full[s], kb, ca,
                                     m_tile * 128 + cfg.a.row_off, cb, n_tile * NT + cfg.b.row_off);
      ++issued;
    }
    *(volatile uint32_t*)issued_s = issued;
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    constexpr uint32_t id = idesc_f16(128, NT, BF16, false);
    constexpr uint32_t idn = idesc_f16(128, NT, BF16, false, true);
    constexpr MmaSchedule<NPLA, NPLB, NACC> S{};
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&full[s], ph, cfg.err, TC_ERR_FULL_WAIT, cfg.wait) || *(volatile uint32_t*)abort_flag) {
        *(volatile uint32_t*)abort_flag = 1;
        break;
      }
      tc_fence_after();
      // descriptors of the stage's first A / B rows; a plane or K offset
      // adds (bytes >> 4) to the start-address field (no carry: < 256 KB)
      const uint64_t da0 = smem_desc(smem_u32(sA + s * G::A_STAGE), G::SWZ);
      const uint64_t db0 = smem_desc(smem_u32(sB + s * G::B_STAGE), G::SWZ);
      const uint32_t acc0 = kb ? 1u : 0u;
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
        for (int o = 0; o < S.n; ++o) {
          const MmaOp op = S.ops[o];
          const uint64_t da = da0 + (uint64_t)((op.ap * G::A_PLANE + ks * 32) >> 4);
          const uint64_t db = db0 + (uint64_t)((op.bp * G::B_PLANE + ks * 32) >> 4);
          const uint32_t accum = (ks > 0 || !op.first) ? 1u : acc0;
          const uint32_t d = tmem + (uint32_t)(op.dsel * NT);
          mma_f16(d, da, db, op.negb ? idn : id, accum);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accf);  // fires once every MMA above has completed (also on abort)
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;             // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;   // which half of the NT columns
    const int row = m_tile * 128 + q * 32 + lane;
    int ea, ebp[2];
    tile_exps<NT>(cfg, ca, cb, row, n_tile, half, lane, ea, ebp);
    typename Epi::State st;
    epi.prefetch(st, batch, row, n_tile * NT + half * 16);
    bool ok = mbar_wait(accf, 0, cfg.err, TC_ERR_ACC_WAIT, cfg.wait);
    ok = __all_sync(0xffffffffu, ok && !*(volatile uint32_t*)abort_flag);  // warp-uniform for tcgen05.ld
    tc_fence_after();
    if (ok) {
      epi.begin(st);
      const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c = half; c < NT / 16; c += 2)
        epi_slice<NT, NACC>(epi, st, cfg, tl, c, half, batch, row, n_tile, ea, ebp);
      epi.end(st, batch);
    }
    tc_fence_before();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*(volatile uint32_t*)abort_flag) {
      // drain: wait (bounded) for the last load of every stage, so no copy
      // lands in shared memory after the CTA has exited
      const int issued = (int)*(volatile uint32_t*)issued_s;
      for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
        if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, cfg.err, TC_ERR_DRAIN)) break;
      }
    }
    // every MMA issued has completed before TMEM is freed (the epilogue's
    // own wait may have given up early)
    mbar_wait(accf, 0, cfg.err, TC_ERR_DRAIN);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

// Persistent variant for short contractions (K of a few hundred), where the
// epilogue costs as much as the MMAs: one CTA per SM walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... (same tile order as the one-tile
// kernel's grid: n fastest, then m, then batch).  TMEM holds NSETS
// accumulator sets of 2 NACC NT columns.  With two, the MMA warp fills one
// while the epilogue warps drain the other; with one (128-wide tiles, whose
// MMAs read half the shared-memory bytes per flop of 64-wide ones), the
// MMAs of a tile wait for the epilogue of the previous one while the copy
// ring already fills with the next tile's operands.  The ring runs on
// across tiles either way.
//   full[s] / empty[s]   copy ring (producer <-> MMA)
//   tfull[b]             MMA -> epilogue: accumulator set b is complete
//   tempty[b]            epilogue -> MMA: set b has been read (8 warp arrivals)
// Every wait is bounded; on expiry the error word is set, every role leaves
// its loop, copies still in flight are waited for and TMEM is freed.
template <int NT, int KC, int NPLA, int NPLB, int STAGES, bool BF16, int NACC, class Epi, int NSETS = 2>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_persistent_kernel(PlaneImg ga, PlaneImg gb, GemmCfg cfg, Epi epi, int n_tiles, int m_tiles,
                              int total_tiles) {
  using G = TileGeom<NT, KC, NPLA, NPLB>;
  static_assert(NSETS == 1 || NSETS == 2, "one or two accumulator sets");
  static_assert(NT % 16 == 0 && NT >= 32 && NT <= 256 && NSETS * 2 * NACC * NT <= 512,
                "the accumulator sets must fit TMEM");
  if (cfg.err && *(volatile unsigned*)cfg.err) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * G::A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * G::B_STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  uint32_t* abort_flag = tslot + 1;
  uint32_t* issued_s = tslot + 2;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (cfg.K + KC - 1) / KC;
  constexpr uint32_t SET = 2 * NACC * NT;  // D0_re | D0_im | D1_re | D1_im [| D2_re | D2_im]
  constexpr uint32_t TCOLS = tmem_alloc_cols(NSETS * SET);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NSETS; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *issued_s = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  volatile uint32_t* abort_v = abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- copy producer
    uint32_t g = 0;
    for (int t = blockIdx.x; t < total_tiles && !*abort_v; t += gridDim.x) {
      const TileIdx ti = tile_at(t, n_tiles, m_tiles, cfg);
      const int n_tile = ti.n_tile, m_tile = ti.m_tile, batch = ti.batch;
      if (epi.skip_tile(m_tile, n_tile, batch)) continue;
      const int ca = cfg.a.coord(batch), cb = cfg.b.coord(batch);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % STAGES);
        const uint32_t ph = (g / STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, cfg.err, TC_ERR_EMPTY_WAIT, cfg.wait) || *abort_v) {
          *abort_v = 1;
          break;
        }
        mbar_arrive_expect_tx(&full[s], G::STAGE);
        load_stage<NT, KC, NPLA, NPLB>(ga, gb, sA + s * G::A_STAGE, sB + s * G::B_STAGE, &full[s], kb, ca,
                                       m_tile * 128 + cfg.a.row_off, cb, n_tile * NT + cfg.b.row_off);
        *(volatile uint32_t*)issued_s = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    constexpr uint32_t id = idesc_f16(128, NT, BF16, false);
    constexpr uint32_t idn = idesc_f16(128, NT, BF16, false, true);
    constexpr MmaSchedule<NPLA, NPLB, NACC> S{};
    uint32_t g = 0, it = 0;
    for (int t = blockIdx.x; t < total_tiles && !*abort_v; t += gridDim.x) {
      const TileIdx ti = tile_at(t, n_tiles, m_tiles, cfg);
      const int n_tile = ti.n_tile, m_tile = ti.m_tile, batch = ti.batch;
      if (epi.skip_tile(m_tile, n_tile, batch)) continue;
      const uint32_t buf = it % NSETS, use = it / NSETS;
      if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, cfg.err, TC_ERR_ACC_WAIT, cfg.wait) || *abort_v) {
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      const uint32_t dset = tmem + buf * SET;
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % STAGES);
        const uint32_t ph = (g / STAGES) & 1;
        if (!mbar_wait(&full[s], ph, cfg.err, TC_ERR_FULL_WAIT, cfg.wait) || *abort_v) {
          *abort_v = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t da0 = smem_desc(smem_u32(sA + s * G::A_STAGE), G::SWZ);
        const uint64_t db0 = smem_desc(smem_u32(sB + s * G::B_STAGE), G::SWZ);
        const uint32_t acc0 = kb ? 1u : 0u;
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
          for (int o = 0; o < S.n; ++o) {
            const MmaOp op = S.ops[o];
            const uint64_t da = da0 + (uint64_t)((op.ap * G::A_PLANE + ks * 32) >> 4);
            const uint64_t db = db0 + (uint64_t)((op.bp * G::B_PLANE + ks * 32) >> 4);
            const uint32_t accum = (ks > 0 || !op.first) ? 1u : acc0;
            mma_f16(dset + (uint32_t)(op.dsel * NT), da, db, op.negb ? idn : id, accum);
          }
        }
        mma_commit(&empty[s]);
      }
      if (!ok) break;
      mma_commit(&tfull[buf]);
      ++it;
    }
    mma_commit(done);  // fires once every MMA issued above has completed
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;             // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;   // which half of the NT columns
    uint32_t it = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
      const TileIdx ti = tile_at(t, n_tiles, m_tiles, cfg);
      const int n_tile = ti.n_tile, m_tile = ti.m_tile, batch = ti.batch;
      if (epi.skip_tile(m_tile, n_tile, batch)) continue;
      const uint32_t buf = it % NSETS, use = it / NSETS;
      const int ca = cfg.a.coord(batch), cb = cfg.b.coord(batch);
      const int row = m_tile * 128 + q * 32 + lane;
      int ea, ebp[2];
      tile_exps<NT>(cfg, ca, cb, row, n_tile, half, lane, ea, ebp);
      typename Epi::State st;
      epi.prefetch(st, batch, row, n_tile * NT + half * 16);
      bool ok = mbar_wait(&tfull[buf], use & 1, cfg.err, TC_ERR_ACC_WAIT, cfg.wait);
      ok = __all_sync(0xffffffffu, ok && !*abort_v);  // warp-uniform for tcgen05.ld
      if (!ok) {
        if (lane == 0) *abort_v = 1;
        break;
      }
      tc_fence_after();
      epi.begin(st);
      const uint32_t tl = tmem + buf * SET + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c = half; c < NT / 16; c += 2)
        epi_slice<NT, NACC>(epi, st, cfg, tl, c, half, batch, row, n_tile, ea, ebp);
      epi.end(st, batch);
      // this warp is done reading set buf: hand it back to the MMA warp
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      ++it;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*abort_v) {
      // drain: wait (bounded) for the last load of every stage, so no copy
      // lands in shared memory after the CTA has exited
      const uint32_t issued = *(volatile uint32_t*)issued_s;
      for (uint32_t g = issued > (uint32_t)STAGES ? issued - STAGES : 0; g < issued; ++g) {
        if (!mbar_wait(&full[g % STAGES], (g / STAGES) & 1, cfg.err, TC_ERR_DRAIN)) break;
      }
    }
    mbar_wait(done, 0, cfg.err, TC_ERR_DRAIN);  // every MMA has completed
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

// Persistent variant with the A operand resident in shared memory, for
// short contractions (K <= NKA * KC) whose A tile serves many output tiles
// (step i: one 128 x N_v tile of the tau blocks serves all N_v^2 / NT
// column tiles of its batch).  CTA b walks a contiguous range of tiles (n
// fastest), loads the whole-K A tile once per (m tile, batch) and streams
// only B through the ring; TMEM holds two accumulator sets as in
// tc_gemm_persistent_kernel.  Not for epilogues that skip tiles.
//   afull   producer -> MMA: the resident A tile has landed
//   afree   MMA -> producer: every MMA reading the resident A has completed
template <int NT, int KC, int NPLA, int NPLB, int NKA, int STAGES, bool BF16, int NACC, class Epi>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_ares_kernel(PlaneImg ga, PlaneImg gb, GemmCfg cfg, Epi epi, int n_tiles, int m_tiles,
                        int total_tiles) {
  using G = TileGeom<NT, KC, NPLA, NPLB>;
  static_assert(NT % 16 == 0 && NT >= 32 && 4 * NACC * NT <= 512, "two accumulator sets must fit TMEM");
  if (cfg.err && *(volatile unsigned*)cfg.err) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + NKA * G::A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * G::B_STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* afull = tempty + 2;
  uint64_t* afree = afull + 1;
  uint64_t* done = afree + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  uint32_t* abort_flag = tslot + 1;
  uint32_t* issued_s = tslot + 2;
  uint32_t* aloads_s = tslot + 3;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (cfg.K + KC - 1) / KC;  // <= NKA, checked by the host
  constexpr uint32_t SET = 2 * NACC * NT;
  constexpr uint32_t TCOLS = tmem_alloc_cols(2 * SET);
  const int per = (total_tiles + (int)gridDim.x - 1) / (int)gridDim.x;
  const int t_begin = (int)blockIdx.x * per;
  const int t_end = min(total_tiles, t_begin + per);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    mbar_init(afull, 1);
    mbar_init(afree, 1);
    mbar_init(done, 1);
    *abort_flag = 0;
    *issued_s = 0;
    *aloads_s = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  volatile uint32_t* abort_v = abort_flag;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- copy producer
    uint32_t g = 0, reloads = 0;
    int key = -1;
    for (int t = t_begin; t < t_end && !*abort_v; ++t) {
      const int n_tile = t % n_tiles, rest = t / n_tiles, m_tile = rest % m_tiles, batch = rest / m_tiles;
      if (rest != key) {
        // the previous A tile is overwritten only after its last MMA completed
        if (reloads > 0 && !mbar_wait(afree, (reloads - 1) & 1, cfg.err, TC_ERR_EMPTY_WAIT, cfg.wait)) {
          *abort_v = 1;
          break;
        }
        const int ca = cfg.a.coord(batch);
        mbar_arrive_expect_tx(afull, nk * G::A_STAGE);
        for (int kb = 0; kb < nk; ++kb)
          load_planes<NPLA, 128>(ga, sA + kb * G::A_STAGE, afull, kb, ca, m_tile * 128 + cfg.a.row_off);
        ++reloads;
        *(volatile uint32_t*)aloads_s = reloads;
        key = rest;
      }
      const int cb = cfg.b.coord(batch);
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % STAGES);
        const uint32_t ph = (g / STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, cfg.err, TC_ERR_EMPTY_WAIT, cfg.wait) || *abort_v) {
          *abort_v = 1;
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[s], G::B_STAGE);
        load_planes<NPLB, NT>(gb, sB + s * G::B_STAGE, &full[s], kb, cb, n_tile * NT + cfg.b.row_off);
        *(volatile uint32_t*)issued_s = g + 1;
      }
      if (!ok) break;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    constexpr uint32_t id = idesc_f16(128, NT, BF16, false);
    constexpr uint32_t idn = idesc_f16(128, NT, BF16, false, true);
    constexpr MmaSchedule<NPLA, NPLB, NACC> S{};
    uint32_t g = 0, it = 0, reloads = 0;
    int key = -1;
    for (int t = t_begin; t < t_end && !*abort_v; ++t) {
      const int rest = t / n_tiles;
      if (rest != key) {
        if (!mbar_wait(afull, reloads & 1, cfg.err, TC_ERR_FULL_WAIT, cfg.wait) || *abort_v) {
          *abort_v = 1;
          break;
        }
        ++reloads;
        key = rest;
      }
      const uint32_t buf = it & 1, use = it >> 1;
      if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, cfg.err, TC_ERR_ACC_WAIT, cfg.wait) || *abort_v) {
        *abort_v = 1;
        break;
      }
      tc_fence_after();
      const uint32_t dset = tmem + buf * SET;
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % STAGES);
        const uint32_t ph = (g / STAGES) & 1;
        if (!mbar_wait(&full[s], ph, cfg.err, TC_ERR_FULL_WAIT, cfg.wait) || *abort_v) {
          *abort_v = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t da0 = smem_desc(smem_u32(sA + kb * G::A_STAGE), G::SWZ);
        const uint64_t db0 = smem_desc(smem_u32(sB + s * G::B_STAGE), G::SWZ);
        const uint32_t acc0 = kb ? 1u : 0u;
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
          for (int o = 0; o < S.n; ++o) {
            const MmaOp op = S.ops[o];
            const uint64_t da = da0 + (uint64_t)((op.ap * G::A_PLANE + ks * 32) >> 4);
            const uint64_t db = db0 + (uint64_t)((op.bp * G::B_PLANE + ks * 32) >> 4);
            const uint32_t accum = (ks > 0 || !op.first) ? 1u : acc0;
            mma_f16(dset + (uint32_t)(op.dsel * NT), da, db, op.negb ? idn : id, accum);
          }
        }
        mma_commit(&empty[s]);
      }
      if (!ok) break;
      mma_commit(&tfull[buf]);
      ++it;
      if (t + 1 >= t_end || (t + 1) / n_tiles != key) mma_commit(afree);  // last tile on this A
    }
    mma_commit(done);  // fires once every MMA issued above has completed
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    uint32_t it = 0;
    for (int t = t_begin; t < t_end; ++t) {
      const int n_tile = t % n_tiles, rest = t / n_tiles, m_tile = rest % m_tiles, batch = rest / m_tiles;
      const uint32_t buf = it & 1, use = it >> 1;
      const int ca = cfg.a.coord(batch), cb = cfg.b.coord(batch);
      const int row = m_tile * 128 + q * 32 + lane;
      int ea, ebp[2];
      tile_exps<NT>(cfg, ca, cb, row, n_tile, half, lane, ea, ebp);
      typename Epi::State st;
      epi.prefetch(st, batch, row, n_tile * NT + half * 16);
      bool ok = mbar_wait(&tfull[buf], use & 1, cfg.err, TC_ERR_ACC_WAIT, cfg.wait);
      ok = __all_sync(0xffffffffu, ok && !*abort_v);
      if (!ok) {
        if (lane == 0) *abort_v = 1;
        break;
      }
      tc_fence_after();
      epi.begin(st);
      const uint32_t tl = tmem + buf * SET + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c = half; c < NT / 16; c += 2)
        epi_slice<NT, NACC>(epi, st, cfg, tl, c, half, batch, row, n_tile, ea, ebp);
      epi.end(st, batch);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      ++it;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*abort_v) {
      // drain: the last load of every ring stage and the last A tile
      const uint32_t issued = *(volatile uint32_t*)issued_s;
      for (uint32_t g = issued > (uint32_t)STAGES ? issued - STAGES : 0; g < issued; ++g) {
        if (!mbar_wait(&full[g % STAGES], (g / STAGES) & 1, cfg.err, TC_ERR_DRAIN)) break;
      }
      const uint32_t al = *(volatile uint32_t*)aloads_s;
      if (al > 0) mbar_wait(afull, (al - 1) & 1, cfg.err, TC_ERR_DRAIN);
    }
    mbar_wait(done, 0, cfg.err, TC_ERR_DRAIN);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

}  // namespace tc
}  // namespace distil
