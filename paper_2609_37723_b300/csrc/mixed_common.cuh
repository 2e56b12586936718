// Pieces shared by the mixed-precision (split 16-bit, tensor-core) paths:
// split schemes, per-row power-of-two exponents, the row-splitting kernel
// and the GEMM epilogues.  Element-wise work runs in FP32 instructions on
// double-float values (df.cuh); FP64 is used only for a handful of values
// per block.
//
// Split schemes.  A row of an operand with max |x| < 2^e is represented as
//  * fixed-point slices: t = x 2^(H-e) = hi + 2^-W mid + 2^-2W lo with hi,
//    mid, lo integers (|hi| <= 2^H, |mid|, |lo| <= 2^(W-1)), exact in the
//    16-bit type (FP16: W = 11, H <= 11; BF16: W = 8, H <= 7).  Products of
//    integer slices are integers, which the tensor core's FP32 accumulation
//    adds exactly, whatever its rounding, while the partial sums stay below
//    2^24; each weight class gets its own TMEM accumulator pair:
//      class 0  hi*hi                     (exact)
//      class 1  hi*mid + mid*hi           (exact while below 2^24)
//      class 2  hi*lo, mid*mid, lo*hi [, lo*mid, mid*lo]   (pre-scaled by
//               2^-W, so fractional: inexact, but ~2^-11 of class 1)
//    With two pairs classes 1 and 2 share one accumulator, whose rounding
//    then drifts with the number of accumulated MMAs (measured ~2.5e-8 of
//    the accumulator per MMA): fine for K <= N_v, not for longer K.  The
//    terms dropped by the 6-product scheme (mid*lo, lo*mid, lo*lo) are of
//    relative size 2^-(W+2+2H) per product, independent of how many bits lo
//    keeps; the 8-product scheme keeps mid*lo and lo*mid (dropping
//    2^-(2W+2+2H)).  Choices, from an emulation of the split on full-size
//    rows and the measured parity:
//      mode contractions (K <= 4 N_v)  H = 10, 6 products, three pairs for
//                                      K = 4 N_v, two for K = N_v
//      elementals (4096-long K chunks) H = 8, 8 products, three pairs
//    A pieces: hi, mid, lo 2^-W (3) or hi, mid, mid 2^-W, lo 2^-W (4).
//    B pieces: hi, mid, mid 2^-W, lo 2^-W.
//  * floating pieces (FP16X3): t = x 2^(14-e) = h + l, h = fp16(t),
//    l = fp16(t - h); accumulation rounding is not exact.
#pragma once
#include <cuda_bf16.h>
#include <type_traits>
#include <utility>
#include <cuda_fp16.h>

#include "common.cuh"
#include "df.cuh"
#include "tc.cuh"
#include "tc_host.cuh"

namespace distil {

struct Scheme {
  bool bf16, fixed;
  int H, W;    // fixed point: t = x 2^(H - e), slices of W bits; floating: H = 14
  int na, nb;  // pieces of the A / B operand
  int nprod;
  int pa[8], pb[8], acc[8];
  float w1;    // weight of the second accumulator (2^-W)
  int shift;   // D *= 2^(eA + eB - shift), shift = 2H
};

inline Scheme scheme_of(int mode) {
  if (mode == DISTIL_MIXED_FP16X6)
    return Scheme{false, true, 10, 11, 3, 4, 6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 3, 2, 0}, {0, 1, 1, 1, 1, 1},
                  1.f / 2048.f, 20};
  if (mode == DISTIL_MIXED_BF16X6)
    return Scheme{true, true, 7, 8, 3, 4, 6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 3, 2, 0}, {0, 1, 1, 1, 1, 1},
                  1.f / 256.f, 14};
  if (mode == DISTIL_MIXED_BF16X3)
    return Scheme{true, true, 7, 8, 2, 2, 3, {0, 0, 1}, {0, 1, 0}, {0, 1, 1}, 1.f / 256.f, 14};
  return Scheme{false, false, 14, 0, 2, 2, 3, {0, 0, 1}, {0, 1, 0}, {0, 1, 1}, 1.f, 28};  // FP16X3
}

// The FP16X6 elementals (K = 3 V3 in 4096-long chunks) use 4 x 4 pieces
// and eight products (the third-order lo*mid and mid*lo kept) with an
// 8-bit leading slice: the hi*mid + mid*hi sums of a chunk stay below 2^24
// and add exactly in their own accumulator, and the dropped terms (lo*lo,
// 2^-(2W+2+2H)) are far below the target.  Other modes use their scheme.
inline Scheme elementals_scheme_of(int mode) {
  if (mode == DISTIL_MIXED_FP16X6)
    return Scheme{false, true, 8, 11, 4, 4, 8, {0, 0, 1, 0, 3, 1, 3, 2}, {0, 1, 0, 3, 0, 2, 2, 3},
                  {0, 1, 1, 2, 2, 2, 2, 2}, 1.f / 2048.f, 16};
  return scheme_of(mode);
}

inline void fill_products(tc::GemmCfg& cfg, const Scheme& s) {
  cfg.nprod = s.nprod;
  for (int i = 0; i < s.nprod; ++i) {
    cfg.pa[i] = s.pa[i];
    cfg.pb[i] = s.pb[i];
    cfg.acc[i] = s.acc[i];
  }
  cfg.w1 = s.w1;
  cfg.shift = s.shift;
}

// Exponent e with max |x| < 2^e (0 for an all-zero row).
__device__ __forceinline__ int row_exponent(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 0;
  int e;
  frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// Slice width of the fixed-point pieces: 11 bits in FP16, 8 in BF16.
template <bool BF16>
struct SliceBits {
  static constexpr int W = BF16 ? 8 : 11;
};

// Exact scaling by 2^n as two power-of-two factors, each in the normal
// range for |n| <= 252 (the row exponents here stay far inside that).
struct Pow2 {
  float a, b;
};
__device__ __forceinline__ Pow2 pow2_pair(int n) {
  const int h = n / 2;
  return Pow2{tc::pow2f(h), tc::pow2f(n - h)};
}
__device__ __forceinline__ float scale2(float x, Pow2 s) { return (x * s.a) * s.b; }

// NPC pieces of the double-float x for a row with exponent e and leading
// slice width H (scheme notes above), given s = 2^(H - e) (pow2_pair,
// computed once per row), in FP32 instructions: scaling by powers of two is
// exact, t.hi - rint(t.hi) is exact, and adding t.lo to that remainder
// rounds far below the last slice.
template <bool BF16, bool FIXED, int NPC>
__device__ __forceinline__ void make_pieces(DF x, Pow2 s, typename tc::Piece<BF16>::T (&p)[NPC]) {
  using PC = tc::Piece<BF16>;
  constexpr int W = SliceBits<BF16>::W;
  if constexpr (FIXED) {
    constexpr float sw = (float)(1 << W), isw = 1.f / (float)(1 << W);
    const float th = scale2(x.hi, s), tl = scale2(x.lo, s);
    const float hi = rintf(th);
    const float r1 = __fmul_rn(__fadd_rn(__fsub_rn(th, hi), tl), sw);
    const float mid = rintf(r1);
    const float lo = rintf(__fmul_rn(__fsub_rn(r1, mid), sw));
    p[0] = PC::from(hi);
    if constexpr (NPC >= 2) p[1] = PC::from(mid);
    if constexpr (NPC == 3) p[2] = PC::from(lo * isw);
    if constexpr (NPC == 4) {
      p[2] = PC::from(mid * isw);
      p[3] = PC::from(lo * isw);
    }
  } else {
    float t = scale2(x.hi, s) + scale2(x.lo, s);
#pragma unroll
    for (int i = 0; i < NPC; ++i) {
      p[i] = PC::from(t);
      t -= PC::to(p[i]);
    }
  }
}

// Pieces of element v at K index k of row rr of coordinate c into the 2 NPC
// planes of img: piece i in the planes 2 ((i + ROT) mod NPC) + re/im (ROT = 2
// with four pieces stores them in the order mid', lo, hi, mid, for the
// two-pass contractions).  Lanes with consecutive k fill whole 32-byte rows
// of a K block together.
template <bool BF16, bool FIXED, int NPC, int ROT = 0>
__device__ __forceinline__ void store_pieces_at(typename tc::Piece<BF16>::T* out, long long ps, const CDF& v, Pow2 sc) {
  using P16 = typename tc::Piece<BF16>::T;
  P16 pr[NPC], pi[NPC];
  make_pieces<BF16, FIXED, NPC>(v.re, sc, pr);
  make_pieces<BF16, FIXED, NPC>(v.im, sc, pi);
#pragma unroll
  for (int i = 0; i < NPC; ++i) {
    const int slot = (i + ROT) % NPC;
    out[(2 * slot) * ps] = pr[i];
    out[(2 * slot + 1) * ps] = pi[i];
  }
}
template <bool BF16, bool FIXED, int NPC, int ROT = 0>
__device__ __forceinline__ void store_pieces(const tc::PlaneImg& img, long long c, long long rr, int k, const CDF& v,
                                             Pow2 sc) {
  using P16 = typename tc::Piece<BF16>::T;
  store_pieces_at<BF16, FIXED, NPC, ROT>(reinterpret_cast<P16*>(img.base) + img.index(c, 0, rr, k), img.rows_pad * 16,
                                         v, sc);
}

// Two 16-bit values packed as one 32-bit word (a in the low half).
template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}
// The three fixed-point pieces (hi, mid, lo 2^-W) of two double-floats x0,
// x1 scaled by one power of two s in FP32's normal range, as packed pairs:
// the values make_pieces<BF16, true, 3> gives with pow2_pair scaling (the
// power-of-two products are exact either way), converted two at a time.
template <bool BF16>
__device__ __forceinline__ void pieces3_pair(DF x0, DF x1, float s, uint32_t& w_hi, uint32_t& w_mid, uint32_t& w_lo) {
  constexpr int W = SliceBits<BF16>::W;
  constexpr float sw = (float)(1 << W), isw = 1.f / (float)(1 << W);
  const float th0 = x0.hi * s, tl0 = x0.lo * s, th1 = x1.hi * s, tl1 = x1.lo * s;
  const float hi0 = rintf(th0), hi1 = rintf(th1);
  const float r0 = __fmul_rn(__fadd_rn(__fsub_rn(th0, hi0), tl0), sw);
  const float r1 = __fmul_rn(__fadd_rn(__fsub_rn(th1, hi1), tl1), sw);
  const float mid0 = rintf(r0), mid1 = rintf(r1);
  const float lo0 = rintf(__fmul_rn(__fsub_rn(r0, mid0), sw)), lo1 = rintf(__fmul_rn(__fsub_rn(r1, mid1), sw));
  w_hi = pack2<BF16>(hi0, hi1);
  w_mid = pack2<BF16>(mid0, mid1);
  w_lo = pack2<BF16>(lo0 * isw, lo1 * isw);
}

// A source may bind a row once (Src::row(r), returning an object with
// operator()(k) and approx(k)) so that the per-row part of its indexing
// runs once per row instead of once per element; otherwise bind_row wraps
// Src::operator()(r, k).
template <class S, class = void>
struct has_row : std::false_type {};
template <class S>
struct has_row<S, std::void_t<decltype(std::declval<const S&>().row(0LL))>> : std::true_type {};
template <class Src>
struct RowOf {
  const Src* src;
  long long r;
  __device__ __forceinline__ CDF operator()(int k) const { return (*src)(r, k); }
  __device__ __forceinline__ float2 approx(int k) const { return src->approx(r, k); }
};
template <class Src>
__device__ __forceinline__ auto bind_row(const Src& src, long long r) {
  if constexpr (has_row<Src>::value)
    return src.row(r);
  else
    return RowOf<Src>{&src, r};
}

// Optional cap on a row's scaled 2-norm: with norm_bits > 0 the exponent is
// raised until 2^(H - e) ||x|| <= 2^norm_bits (ss = ||x||^2, padded for its
// FP32 rounding).  Two rows capped at 2^11 keep every leading-slice sum
// |sum_k hi_a hi_b| <= ||hi_a|| ||hi_b|| below 2^24 whatever the K and
// however aligned the rows (a coherent sum such as sum_x |v(x)|^2 reaches
// that bound long before a random-sign one), so the class-0 accumulation
// stays exact.  Off (0) for operands whose rows are known to sum with random
// signs.
__device__ __forceinline__ int norm_capped_exponent(int e, float ss, int H, int norm_bits) {
  if (norm_bits <= 0 || !(ss > 0.f)) return e;
  int en;
  frexpf(sqrtf(ss) * (1.f + 1.f / 4096.f), &en);  // ||x|| < 2^en
  const int ec = H - norm_bits + en;
  return ec > e ? ec : e;
}

// A source may give each row its own norm cap (Src::norm_bits(r), 0 = none)
// in place of the split's one value: only rows that can sum coherently
// against the other operand need one.
template <class S, class = void>
struct has_norm_bits : std::false_type {};
template <class S>
struct has_norm_bits<S, std::void_t<decltype(std::declval<const S&>().norm_bits(0LL))>> : std::true_type {};
template <class Src>
__device__ __forceinline__ int row_norm_bits(const Src& src, long long r, int dflt) {
  if constexpr (has_norm_bits<Src>::value)
    return src.norm_bits(r);
  else
    return dflt;
}

// Split rows of a complex operand into 2*NPC planes with a per-row exponent.
// Global row r = coord * img.rows + rr goes to plane image img (tc_gemm.cuh:
// PlaneImg; plane 2 i + re/im holds piece i) at coordinate coord, row rr,
// and exps[r]; the K elements of the last K block past img.K are stored as
// zeros.  Optionally the row's 2-norm (with a small safety margin) goes
// into norms[r].  One warp per row: pass 1 finds max |re|, |im| over the
// row, pass 2 writes the pieces.  Src::operator()(r, k) returns the element
// as a complex double-float, Src::approx(r, k) an FP32 estimate of it.
template <bool BF16, bool FIXED, int NPC, class Src, int ROT = 0>
__global__ void __launch_bounds__(256) split_rows_kernel(Src src, long long nrows, tc::PlaneImg img, int H,
                                                         int* __restrict__ exps, float* __restrict__ norms,
                                                         int norm_bits) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int K = img.K, Kp = img.kblocks * 16;
  const auto row = bind_row(src, r);
  float m = 0.f, ss = 0.f;
  for (int k = lane; k < K; k += 32) {
    const float2 v = row.approx(k);  // FP32 estimate: enough for the exponent and the norm
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    ss = fmaf(v.x, v.x, fmaf(v.y, v.y, ss));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  // the FP32 estimate may sit slightly below the true magnitude: pad by 2^-16
  const int e =
      norm_capped_exponent(row_exponent(m * (1.f + 1.f / 65536.f)), ss, H, row_norm_bits(src, r, norm_bits));
  if (lane == 0) {
    exps[r] = e;
    if (norms) norms[r] = sqrtf(ss) * (1.f + 1e-5f);
  }
  const Pow2 sc = pow2_pair(H - e);
  const long long coord = r / img.rows, rr = r % img.rows;
  // k = lane + 32 u: each step moves two K blocks on; the swizzle half and
  // k & 7 stay those of the lane
  using P16 = typename tc::Piece<BF16>::T;
  P16* out = reinterpret_cast<P16*>(img.base) + img.index(coord, 0, rr, lane);
  const long long ps = img.rows_pad * 16, step = 2 * (long long)img.ptot * ps;
  for (int k = lane; k < Kp; k += 32, out += step)
    store_pieces_at<BF16, FIXED, NPC, ROT>(out, ps, k < K ? row(k) : cdf_zero(), sc);
}

// Long rows (K <= 512 PER): one block of 512 threads per row, each thread
// holding PER elements in registers, so every element is formed once and
// the exponent comes from the exact maximum.
template <bool BF16, bool FIXED, int NPC, int PER, class Src, int ROT = 0>
__global__ void __launch_bounds__(512) split_rows_cached_kernel(Src src, tc::PlaneImg img, int H,
                                                                int* __restrict__ exps, float* __restrict__ norms,
                                                                int norm_bits) {
  __shared__ float red_m[16], red_s[16];
  __shared__ int sh_e;
  const long long r = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int K = img.K, Kp = img.kblocks * 16;
  const auto row = bind_row(src, r);
  CDF v[PER];
  float m = 0.f, ss = 0.f;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int k = threadIdx.x + 512 * u;
    v[u] = k < K ? row(k) : cdf_zero();
    m = fmaxf(m, fmaxf(fabsf(v[u].re.hi), fabsf(v[u].im.hi)));
    ss = fmaf(v[u].re.hi, v[u].re.hi, fmaf(v[u].im.hi, v[u].im.hi, ss));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if (lane == 0) { red_m[wid] = m; red_s[wid] = ss; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 16; ++w) { m = fmaxf(m, red_m[w]); ss += red_s[w]; }
    sh_e =
        norm_capped_exponent(row_exponent(m * (1.f + 1.f / 65536.f)), ss, H, row_norm_bits(src, r, norm_bits));
    exps[r] = sh_e;
    if (norms) norms[r] = sqrtf(ss) * (1.f + 1e-5f);
  }
  __syncthreads();
  const Pow2 sc = pow2_pair(H - sh_e);
  const long long coord = r / img.rows, rr = r % img.rows;
  // k = tid + 512 u: each step moves 32 K blocks on; the swizzle half and
  // k & 7 stay those of the thread
  using P16 = typename tc::Piece<BF16>::T;
  P16* out = reinterpret_cast<P16*>(img.base) + img.index(coord, 0, rr, threadIdx.x);
  const long long ps = img.rows_pad * 16, step = 32 * (long long)img.ptot * ps;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int k = threadIdx.x + 512 * u;
    if (k >= Kp) break;
    store_pieces_at<BF16, FIXED, NPC, ROT>(out + u * step, ps, v[u], sc);
  }
}

// Zero the elements past K in the last K block of every row of a plane
// image whose writer leaves them (the step-i epilogue writes K = 4 N_v
// elements only): one thread per (coordinate, plane, row).
static __global__ void img_zero_kpad_kernel(tc::PlaneImg img) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long rows = (long long)img.coords * img.ptot * img.rows;
  if (t >= rows) return;
  const long long c = t / ((long long)img.ptot * img.rows);
  const int p = (int)((t / img.rows) % img.ptot);
  const long long r = t % img.rows;
  uint16_t* out = reinterpret_cast<uint16_t*>(img.base);
  for (int k = img.K; k < img.kblocks * 16; ++k) out[img.index(c, p, r, k)] = 0;
}

template <bool BF16, bool FIXED, int NPC, class Src, int ROT = 0>
inline int split_rows(distil_ctx* ctx, const char* name, const Src& src, long long nrows, const tc::PlaneImg& img,
                      int H, int* exps, cudaStream_t s, float* norms = nullptr, int norm_bits = 0) {
  if (nrows <= 0) return DISTIL_OK;
  if (img.planes != 2 * NPC || img.ptot != img.planes || img.p0 != 0 || nrows > (long long)img.coords * img.rows ||
      img.kblocks * 16 < img.K) {
    set_error("%s: rows or planes outside the plane image", name);
    return DISTIL_EINVAL;
  }
  const int K = img.K;
  const long long threads = nrows * 32;
  Launch L(ctx, name, s);
  if (K > 2048 && K <= 4096)
    split_rows_cached_kernel<BF16, FIXED, NPC, 8, Src, ROT><<<(unsigned)nrows, 512, 0, s>>>(src, img, H, exps, norms,
                                                                                          norm_bits);
  else if (K > 1024 && K <= 2048)
    split_rows_cached_kernel<BF16, FIXED, NPC, 4, Src, ROT><<<(unsigned)nrows, 512, 0, s>>>(src, img, H, exps, norms,
                                                                                          norm_bits);
  else
    split_rows_kernel<BF16, FIXED, NPC, Src, ROT><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(src, nrows, img,
                                                                                                     H, exps, norms,
                                                                                                     norm_bits);
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

inline int img_zero_kpad(distil_ctx* ctx, const tc::PlaneImg& img, cudaStream_t s) {
  if (img.kblocks * 16 == img.K) return DISTIL_OK;
  const long long rows = (long long)img.coords * img.ptot * img.rows;
  Launch L(ctx, "img_zero_kpad", s);
  img_zero_kpad_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(img);
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

// --------------------------------------------------------------- epilogues
// Column map shared by the epilogues: colmap(c) = (c / cdiv) * cs1 +
// (c % cdiv) * sc, or c * sc when cdiv == 0; with cdiv, columns whose
// c % cdiv >= cvalid are padding and are not stored.
struct ColMap {
  long long sc;
  int cdiv;
  long long cs1;
  int cvalid;
  __device__ __forceinline__ long long operator()(int c) const {
    return cdiv ? (long long)(c / cdiv) * cs1 + (long long)(c % cdiv) * sc : (long long)c * sc;
  }
  __device__ __forceinline__ bool keep(int c) const { return !cdiv || (c % cdiv) < cvalid; }
};

// 16-byte load of a complex double-float (p 16-byte aligned)
__device__ __forceinline__ CDF ld_cdf(const CDF* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return cdf_make(df_make(v.x, v.y), df_make(v.z, v.w));
}

// The GEMM hands the epilogue each value as an unevaluated FP32 pair
// (leading-slice part, cross-term part): D = re0 + re1, im0 + im1.

// out[batch][row * sr + colmap(col)] = D as a complex double-float.
struct EpiStoreCDF : tc::EpiStateless {
  CDF* out;
  long long sb_hi, sb_lo;
  int b_lo;
  long long sr;
  ColMap cm;
  int N;
  __device__ __forceinline__ bool skip_tile(int, int, int) const { return false; }
  __device__ __forceinline__ void operator()(State&, int batch, int row, int col0, const float* re0, const float* re1,
                                             const float* im0, const float* im1) const {
    CDF* base = out + (long long)(batch / b_lo) * sb_hi + (long long)(batch % b_lo) * sb_lo + (long long)row * sr;
    if (!cm.cdiv && cm.sc == 1 && col0 + 16 <= N && !(reinterpret_cast<uintptr_t>(base + col0) & 31)) {
      // 16 contiguous outputs of this row: two per 32-byte store
      CDF* d = base + col0;
#pragma unroll
      for (int e = 0; e < 16; e += 2) {
        const DF r0 = two_sum(re0[e], re1[e]), i0 = two_sum(im0[e], im1[e]);
        const DF r1 = two_sum(re0[e + 1], re1[e + 1]), i1 = two_sum(im0[e + 1], im1[e + 1]);
        const uint32_t w[8] = {__float_as_uint(r0.hi), __float_as_uint(r0.lo), __float_as_uint(i0.hi),
                               __float_as_uint(i0.lo), __float_as_uint(r1.hi), __float_as_uint(r1.lo),
                               __float_as_uint(i1.hi), __float_as_uint(i1.lo)};
        tc::st_global_32B(d + e, w);
      }
      return;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      if (c >= N) break;
      if (cm.keep(c)) base[cm(c)] = cdf_make(two_sum(re0[e], re1[e]), two_sum(im0[e], im1[e]));
    }
  }
};

// out[batch][row * sr + colmap(col)] += D (complex double-float): the
// second pass of a contraction split by accumulator class.
struct EpiAddCDF : tc::EpiStateless {
  CDF* out;
  long long sb_hi, sb_lo;
  int b_lo;
  long long sr;
  ColMap cm;
  int N;
  __device__ __forceinline__ bool skip_tile(int, int, int) const { return false; }
  __device__ __forceinline__ void operator()(State&, int batch, int row, int col0, const float* re0, const float* re1,
                                             const float* im0, const float* im1) const {
    CDF* base = out + (long long)(batch / b_lo) * sb_hi + (long long)(batch % b_lo) * sb_lo + (long long)row * sr;
    // all 16 loads in flight before the first store (the stores could
    // otherwise alias the later loads and serialise the round trips)
    CDF old[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      old[e] = (c < N && cm.keep(c)) ? ld_cdf(base + cm(c)) : cdf_zero();
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      if (c < N && cm.keep(c))
        base[cm(c)] = cdf_add(old[e], cdf_make(two_sum(re0[e], re1[e]), two_sum(im0[e], im1[e])));
    }
  }
};

// out[batch][row][col] = D rounded to complex64 (public split GEMM).
struct EpiStoreC64 : tc::EpiStateless {
  float2* out;
  long long sb;
  long long sr;
  int N;
  __device__ __forceinline__ bool skip_tile(int, int, int) const { return false; }
  __device__ __forceinline__ void operator()(State&, int batch, int row, int col0, const float* re0, const float* re1,
                                             const float* im0, const float* im1) const {
    float2* base = out + (long long)batch * sb + (long long)row * sr;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      if (c >= N) break;
      const DF r = two_sum(re0[e], re1[e]), i = two_sum(im0[e], im1[e]);
      base[c] = make_float2(r.hi, i.hi);
    }
  }
};

}  // namespace distil
