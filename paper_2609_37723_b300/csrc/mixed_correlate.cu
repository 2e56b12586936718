// Mixed-precision correlation matrix: the three mode contractions of
// correlate.cuh on tcgen05 tensor cores with operands split into 16-bit
// pieces with per-row power-of-two exponents (mixed_common.cuh), FP32
// accumulation in TMEM, double-float intermediates between the contractions
// and a double-float dot whose block sums are added into C in FP64.
//
// Every (t, p) is first normalised: tau(t) by 2^-e_tau(t), Phi_snk(t,p) by
// 2^-e_snk, Phi_src(p) by 2^-e_src (exponents of their largest entries), so
// every intermediate stays well inside the FP32 range however fast tau
// decays with t; C picks the factor 2^(3 e_tau + e_snk + e_src) back up in
// FP64.
//
// Per (t, p):
//   split    Aa  rows (a'beta, i')  K i        from Gamma_beta tau[(alpha(beta) i)][(a' i')]
//            tauT rows (b' j')      K (beta j) from tau[(beta j)][(b' j')]
//                                              (b' blocks of N_v rounded up to 8 rows)
//            TcT rows k'            K (c, k)   from the five source blocks T^c[k][k']
//            G   rows (a, (k,j))    K i        from g g g Phi_snk
//   step i   U[a][a'][(i',k)][(beta,j)] = sum_i Aa G, split by the epilogue
//            with the row exponent of the Cauchy-Schwarz bound
//            |U| <= max_beta |Aa row| * max_j |G row|
//   step j   V[a][slot][j'][(i',k)]     = sum_(beta,j) U tauT
//   split    W rows (a, i'<j')      K (c, k)   the source-weighted antisymmetric
//                                              parts w^a_c of V (correlate.cuh)
//   T contr. Z[a][pair][k']         = sum_(c,k) W TcT
//   dot      C_ab = sum_(pair,k') Z^a gamma^b conj(Phi_src~), with
//            gamma^b = g^b_i' g^b_j' g^b_k' the only b-dependence
#include <algorithm>

#include "correlate.cuh"
#include "df.cuh"
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

using tc::PlaneImg;

// ------------------------------------------------------------------ setup
// binary exponent e with |x| < 2^e for the largest |component| of a complex128
// array, from the bit patterns (no FP64 arithmetic)
__device__ __forceinline__ int dbl_exp_bound(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  return ex == 0 ? -1022 : ex - 1022;  // |x| < 2^(ex - 1023 + 1)
}
// exps[i] >= every element's exponent bound of complex128 array i (of
// `count` arrays of `len` values): array i = blockIdx.y, spread over
// gridDim.x blocks that combine with atomicMax into exps[i], which must
// start below -1022 (exp_init_kernel)
__global__ void exp_init_kernel(int* __restrict__ exps, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) exps[i] = -2147483647;
}
__global__ void c128_exp_kernel(const double2* __restrict__ x, long long len, int* __restrict__ exps) {
  const double2* a = x + (long long)blockIdx.y * len;
  int m = -1022;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    m = max(m, max(dbl_exp_bound(a[e].x), dbl_exp_bound(a[e].y)));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&exps[blockIdx.y], m);
}
// exps[i] with max |x| < 2^exps[i] for complex64 array i = blockIdx.y
// (same scheme; the row exponent of the block maximum is monotone in it)
__global__ void c64_exp_kernel(const float2* __restrict__ x, long long len, int* __restrict__ exps) {
  const float2* a = x + (long long)blockIdx.y * len;
  float m = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(a[e].x), fabsf(a[e].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&exps[blockIdx.y], row_exponent(m));
}
// complex128 -> complex double-float, times 2^-e: array y = blockIdx.y of
// `len` values (input stride xs, output stride len) with exponent exps[y]
__global__ void c128_to_cdf_kernel(const double2* __restrict__ x, long long len, long long xs,
                                   const int* __restrict__ exps, CDF* __restrict__ out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= len) return;
  const int y = blockIdx.y;
  const double s = ldexp(1.0, -exps[y]);
  const double2 v = x[y * xs + e];
  out[y * len + e] = cdf_make(df_from_double(v.x * s), df_from_double(v.y * s));
}
__global__ void prof_to_df_kernel(const double* __restrict__ g, long long n, DF* __restrict__ out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) out[e] = df_from_double(g[e]);
}

// ------------------------------------------------------------------ sources
__device__ __forceinline__ CDF cdf_of(float2 x, float s) {
  return cdf_make(df_make(x.x * s, 0.f), df_make(x.y * s, 0.f));
}
struct AaSrc {  // rows (a'*4 + beta)*n + i', K = i
  const float2* tau;
  const int* etau;
  int n;
  __device__ __forceinline__ CDF operator()(long long r, int i) const {
    const int ab = (int)(r / n), ip = (int)(r % n);
    const int ap = ab >> 2, beta = ab & 3, alpha = beta ^ 1;
    // Gamma_{10} = Gamma_{32} = +1, Gamma_{01} = Gamma_{23} = -1
    const float s = (beta & 1) ? -tc::pow2f(-etau[0]) : tc::pow2f(-etau[0]);
    return cdf_of(tau[((long long)alpha * n + i) * 4 * n + ap * n + ip], s);
  }
  __device__ __forceinline__ float2 approx(long long r, int i) const {
    const CDF v = (*this)(r, i);
    return make_float2(v.re.hi, v.im.hi);
  }
};
struct TTSrc {  // rows b' nvp + j' (blocks of nvp >= n rows, the rows past n zero), K = (beta j): tau^T
  const float2* tau;
  const int* etau;
  int n, nvp;
  __device__ __forceinline__ float2 at(long long r, int k) const {
    const int bp = (int)(r / nvp), jp = (int)(r % nvp);
    if (jp >= n) return make_float2(0.f, 0.f);
    const float2 x = tau[(long long)k * 4 * n + (long long)bp * n + jp];
    const float s = tc::pow2f(-etau[0]);
    return make_float2(x.x * s, x.y * s);
  }
  __device__ __forceinline__ CDF operator()(long long r, int k) const { return cdf_of(at(r, k), 1.f); }
  __device__ __forceinline__ float2 approx(long long r, int k) const { return at(r, k); }
};
struct TcSrc {  // rows c*n + k, K = k': T^c[k][k']
  const float2* tau;
  const int* etau;
  int n;
  __device__ __forceinline__ CDF operator()(long long r, int kp) const {
    const int c = (int)(r / n), k = (int)(r % n);
    const long long n4 = 4LL * n;
    const float s = tc::pow2f(-etau[0]);
    if (c == 0) {
      const float2 a = tau[(long long)k * n4 + kp], b = tau[((long long)n + k) * n4 + n + kp];
      return cdf_make(two_sum(a.x * s, b.x * s), two_sum(a.y * s, b.y * s));
    }
    const int mu = (c <= 2) ? 0 : 1;
    const int gp = (c == 1 || c == 3) ? 2 : 3;
    return cdf_of(tau[((long long)mu * n + k) * n4 + gp * n + kp], s);
  }
  __device__ __forceinline__ float2 approx(long long r, int kp) const {
    const CDF v = (*this)(r, kp);
    return make_float2(v.re.hi, v.im.hi);
  }
};
struct TcTSrc {  // rows k', K = (c, k): T^c[k][k'] (TcSrc transposed)
  TcSrc tc;
  __device__ __forceinline__ CDF operator()(long long kp, int kk) const { return tc(kk, (int)kp); }
  __device__ __forceinline__ float2 approx(long long kp, int kk) const { return tc.approx(kk, (int)kp); }
};
// sorted-triple lookup with sign; 0 on a repeated index
__device__ __forceinline__ CDF phi_at(const CDF* phi, int i, int j, int k, DF w) {
  if (i == j || j == k || i == k) return cdf_zero();
  int x = i, y = j, z = k;
  bool neg = false;
  if (x > y) { int t = x; x = y; y = t; neg = !neg; }
  if (y > z) { int t = y; y = z; z = t; neg = !neg; }
  if (x > y) { int t = x; x = y; y = t; neg = !neg; }
  return cdf_scale(phi[triple_rank(x, y, z)], neg ? df_neg(w) : w);
}
struct GSrc {  // rows (qb nb + a) n^2 + k n + j, K = i: g_i g_j g_k Phi_ijk of momentum qb of the batch
  const CDF* phi;  // [qb][T3]
  const DF* g;     // [nb][n]
  int n, nb;
  long long T3;
  __device__ __forceinline__ void unpack(long long r, const CDF*& ph, const DF*& ga, int& k, int& j) const {
    const long long n2 = (long long)n * n;
    const long long ab = r / n2;
    const int qb = (int)(ab / nb), a = (int)(ab - (long long)qb * nb);
    k = (int)((r % n2) / n);
    j = (int)(r % n);
    ph = phi + qb * T3;
    ga = g + (long long)a * n;
  }
  __device__ __forceinline__ CDF operator()(long long r, int i) const {
    const CDF* ph;
    const DF* ga;
    int k, j;
    unpack(r, ph, ga, k, j);
    return phi_at(ph, i, j, k, df_mul(df_mul(ga[i], ga[j]), ga[k]));
  }
  __device__ __forceinline__ float2 approx(long long r, int i) const {
    const CDF* ph;
    const DF* ga;
    int k, j;
    unpack(r, ph, ga, k, j);
    if (i == j || j == k || i == k) return make_float2(0.f, 0.f);
    int x = i, y = j, z = k;
    if (x > y) { int t = x; x = y; y = t; }
    if (y > z) { int t = y; y = z; z = t; }
    if (x > y) { int t = x; x = y; y = t; }
    const float w = ga[i].hi * ga[j].hi * ga[k].hi;
    const CDF p = ph[triple_rank(x, y, z)];
    return make_float2(p.re.hi * w, p.im.hi * w);
  }
};
// mG[a*n + k] = max_j |G row (a, k, j)| (one warp per (a, k)).
__global__ void g_rowmax_kernel(const float* __restrict__ nG, int n, int nb, float* __restrict__ mG) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)nb * n) return;
  const float* g = nG + w * n;
  float m = 0.f;
  for (int j = lane; j < n; j += 32) m = fmaxf(m, g[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) mG[w] = m;
}

// eU[(a*3 + a')*n^2 + i'*n + k] = exponent of max_beta |Aa row (a'beta, i')| * max_j |G row (a, k, j)|,
// a bound on every |U| of that row of the step-i output (Cauchy-Schwarz on the row norms).
__global__ void u_exponent_kernel(const float* __restrict__ nAa, const float* __restrict__ mG, int n, int nb,
                                  int* __restrict__ eU) {
  const long long n2 = (long long)n * n;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= 3LL * nb * n2) return;
  const int ab = (int)(e / n2);  // a*3 + a'
  const int a = ab / 3, ap = ab - 3 * a;
  const int r = (int)(e - ab * n2), ip = r / n, k = r - ip * n;
  float mA = 0.f;
  for (int beta = 0; beta < 4; ++beta) mA = fmaxf(mA, nAa[(ap * 4 + beta) * n + ip]);
  eU[e] = row_exponent(mA * mG[a * n + k] * (1.f + 1e-5f));
}

// Step i epilogue: split U straight from the accumulator pair into the
// A-operand pieces of step j: plane image U, coordinate (a, a'), row (i', k),
// K index (beta, j).
template <bool BF16, bool FIXED, int NPC>
struct EpiSplitU : tc::EpiStateless {
  PlaneImg out;
  const int* eU;
  int n, H;
  // the exponent of U row (row, k) for the k of the warp's first slice,
  // loaded before the accumulator wait (at N_v >= 128 one 128-wide tile
  // has a single k)
  struct State {
    int k, e;
  };
  __device__ __forceinline__ void prefetch(State& st, int batch, int row, int col) const {
    const long long n2 = (long long)n * n;
    st.k = col / n;
    st.e = (row < n && col < n2) ? eU[(long long)(batch >> 2) * n2 + (long long)row * n + st.k] : 0;
  }
  __device__ __forceinline__ void begin(State&) const {}
  __device__ __forceinline__ void end(State&, int) const {}
  __device__ __forceinline__ bool skip_tile(int, int, int) const { return false; }
  // the 2 NPC plane rows of U row ur from K element kk0 (a K block's first):
  // one 32-byte store each, halves in the row's swizzled order
  template <class P16>
  __device__ __forceinline__ void store_row(P16* o, long long ur, int aa, int kk0, int sw,
                                            const uint32_t (&w)[2 * NPC][8]) const {
    P16* d = o + ((out.block(aa, kk0 >> 4, 0) + ur) << 4);
    const long long ps = out.rows_pad * 16;
#pragma unroll
    for (int pl = 0; pl < 2 * NPC; ++pl) {
      uint32_t v[8];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        v[x] = sw ? w[pl][4 + x] : w[pl][x];
        v[4 + x] = sw ? w[pl][x] : w[pl][4 + x];
      }
      tc::st_global_32B(d + pl * ps, v);
    }
  }
  __device__ __forceinline__ void operator()(State& st, int batch, int row, int col0, const float* re0,
                                             const float* re1, const float* im0, const float* im1) const {
    using P16 = typename tc::Piece<BF16>::T;
    const long long n2 = (long long)n * n;
    const int aa = batch >> 2, beta = batch & 3;  // aa = a*3 + a'
    P16* o = reinterpret_cast<P16*>(out.base);
    if ((n & 15) == 0 && col0 + 16 <= (int)n2) {
      // the 16 columns share k and run over 16 consecutive j: one 32-byte
      // row of a K block of the image per plane, assembled in registers
      // (its two 16-byte halves in the row's swizzled order) and written
      // with one 32-byte store
      const int k = col0 / n, j0 = col0 % n;
      const long long ur = (long long)row * n + k;
      const int eu = k == st.k ? st.e : eU[(long long)aa * n2 + ur];
      const Pow2 sc = pow2_pair(H - eu);
      const int sw = (int)(ur >> 2) & 1;  // halves swapped in this row
      uint32_t w[2 * NPC][8];
      if constexpr (FIXED && NPC == 3) {
        if (H - eu >= -126 && H - eu <= 127) {
          // one exact scaling per value, conversions two at a time
          const float s1 = tc::pow2f(H - eu);
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            pieces3_pair<BF16>(two_sum(re0[e], re1[e]), two_sum(re0[e + 1], re1[e + 1]), s1, w[0][e / 2],
                               w[2][e / 2], w[4][e / 2]);
            pieces3_pair<BF16>(two_sum(im0[e], im1[e]), two_sum(im0[e + 1], im1[e + 1]), s1, w[1][e / 2],
                               w[3][e / 2], w[5][e / 2]);
          }
          store_row(o, ur, aa, beta * n + j0, sw, w);
          return;
        }
      }
#pragma unroll
      for (int e = 0; e < 16; e += 2) {
        P16 pr0[NPC], pi0[NPC], pr1[NPC], pi1[NPC];
        make_pieces<BF16, FIXED, NPC>(two_sum(re0[e], re1[e]), sc, pr0);
        make_pieces<BF16, FIXED, NPC>(two_sum(im0[e], im1[e]), sc, pi0);
        make_pieces<BF16, FIXED, NPC>(two_sum(re0[e + 1], re1[e + 1]), sc, pr1);
        make_pieces<BF16, FIXED, NPC>(two_sum(im0[e + 1], im1[e + 1]), sc, pi1);
#pragma unroll
        for (int q = 0; q < NPC; ++q) {
          w[2 * q][e / 2] = (uint32_t)reinterpret_cast<const uint16_t&>(pr0[q]) |
                            ((uint32_t)reinterpret_cast<const uint16_t&>(pr1[q]) << 16);
          w[2 * q + 1][e / 2] = (uint32_t)reinterpret_cast<const uint16_t&>(pi0[q]) |
                                ((uint32_t)reinterpret_cast<const uint16_t&>(pi1[q]) << 16);
        }
      }
      store_row(o, ur, aa, beta * n + j0, sw, w);
      return;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = col0 + e;
      if (c >= (int)n2) break;
      const int k = c / n, j = c % n;
      const long long ur = (long long)row * n + k;
      const Pow2 sc = pow2_pair(H - eU[(long long)aa * n2 + ur]);
      typename tc::Piece<BF16>::T pr[NPC], pi[NPC];
      make_pieces<BF16, FIXED, NPC>(two_sum(re0[e], re1[e]), sc, pr);
      make_pieces<BF16, FIXED, NPC>(two_sum(im0[e], im1[e]), sc, pi);
      P16* d = o + out.index(aa, 0, ur, beta * n + j);
      const long long ps = out.rows_pad * 16;
#pragma unroll
      for (int q = 0; q < NPC; ++q) {
        d[(2 * q) * ps] = pr[q];
        d[(2 * q + 1) * ps] = pi[q];
      }
    }
  }
};

// ------------------------------------------------------------------ dot
// accumulate a * b (double-floats) into the unevaluated pair (s, c)
__device__ __forceinline__ void df_acc_prod(float& s, float& c, DF a, DF b) {
  const DF p = two_prod(a.hi, b.hi);
  const DF t = two_sum(s, p.hi);
  s = t.hi;
  c += t.lo + __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
}

__device__ __forceinline__ CDF ldg_cdf(const CDF* p) {  // p is 16-byte aligned
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return cdf_make(df_make(v.x, v.y), df_make(v.z, v.w));
}

// W^a[pair][(c, k)] = w^a_c[pair][k], the combinations of the antisymmetric
// parts d_s[pair][k] = V^a_{j'i'k} - V^a_{i'j'k} of the sink spin slots s
// that meet source matrix c (correlate.cuh: coefficients -3, -2 on matrix 0,
// +-1 on the others), split into NPC fixed-point pieces with one exponent
// per row (a, pair).  One block per row, thread tid takes k = tid + 256 u.
// Plane image out: coordinate a, row pair, K index c n + k (the elements
// past 5 n in the last K block stored as zeros).
template <bool BF16, bool FIXED, int NPC, int PER>
__global__ void __launch_bounds__(256) split_w_kernel(const CDF* __restrict__ V, int nv, long long P2, int H,
                                                      PlaneImg out, int* __restrict__ exps) {
  using P16 = typename tc::Piece<BF16>::T;
  __shared__ float red[8];
  __shared__ int sh_e;
  const long long r = blockIdx.x;
  const int a = (int)(r / P2);
  const long long pair = r - (long long)a * P2;
  int ip, jp;
  pair_unrank(pair, ip, jp);
  const long long n = nv, n3 = n * n * n;
  const CDF* Va = V + (long long)a * NPAIR * n3;
  const long long o1 = ((long long)jp * n + ip) * n, o2 = ((long long)ip * n + jp) * n;
  CDF w[PER][NSRC];
  float m = 0.f;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int k = threadIdx.x + 256 * u;
    if (k < nv) {
      CDF d[NTERM];
#pragma unroll
      for (int t = 0; t < NTERM; ++t) {
        const CDF* Vs = Va + dot_slot(t) * n3;
        const CDF v1 = ldg_cdf(Vs + o1 + k), v2 = ldg_cdf(Vs + o2 + k);
        d[t] = cdf_make(df_sub_fast(v1.re, v2.re), df_sub_fast(v1.im, v2.im));
      }
      static_assert(dot_coef(0) == -3.0 && dot_coef(1) == -2.0 && dot_src(0) == 0 && dot_src(1) == 0,
                    "source-0 terms");
      static_assert(dot_coef(2) == -1.0 && dot_coef(3) == 1.0 && dot_coef(4) == -1.0 && dot_coef(5) == 1.0,
                    "unit coefficients");
      // w_0 = -3 d_0 - 2 d_1 = -(2 (d_0 + d_1) + d_0); w_c = coef_t d_t for the others
      const DF sr = df_add(d[0].re, d[1].re), si = df_add(d[0].im, d[1].im);
      w[u][0] = cdf_make(df_neg(df_add(df_make(2.f * sr.hi, 2.f * sr.lo), d[0].re)),
                         df_neg(df_add(df_make(2.f * si.hi, 2.f * si.lo), d[0].im)));
#pragma unroll
      for (int t = 2; t < NTERM; ++t)
        w[u][dot_src(t)] = dot_coef(t) > 0 ? d[t] : cdf_make(df_neg(d[t].re), df_neg(d[t].im));
#pragma unroll
      for (int c = 0; c < NSRC; ++c) m = fmaxf(m, fmaxf(fabsf(w[u][c].re.hi), fabsf(w[u][c].im.hi)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < 8; ++i) m = fmaxf(m, red[i]);
    m = fmaxf(m, red[0]);
    sh_e = row_exponent(m * (1.f + 1.f / 65536.f));
    exps[r] = sh_e;
  }
  __syncthreads();
  const Pow2 sc = pow2_pair(H - sh_e);
  P16* o = reinterpret_cast<P16*>(out.base);
  const long long ps = out.rows_pad * 16;  // plane stride in elements
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int k = threadIdx.x + 256 * u;
    if (k >= nv) break;
#pragma unroll
    for (int c = 0; c < NSRC; ++c) {
      P16 pr[NPC], pi[NPC];
      make_pieces<BF16, FIXED, NPC>(w[u][c].re, sc, pr);
      make_pieces<BF16, FIXED, NPC>(w[u][c].im, sc, pi);
      P16* d = o + out.index(a, 0, pair, c * nv + k);
#pragma unroll
      for (int q = 0; q < NPC; ++q) {
        d[(2 * q) * ps] = pr[q];
        d[(2 * q + 1) * ps] = pi[q];
      }
    }
  }
  // zeros past K = NSRC n in the last K block
  for (int kk = NSRC * nv + (int)threadIdx.x; kk < out.kblocks * 16; kk += 256) {
#pragma unroll
    for (int q = 0; q < 2 * NPC; ++q) o[out.index(a, q, pair, kk)] = tc::Piece<BF16>::from(0.f);
  }
}

// Each block leaves its partial sums in part[block][a][b] (FP64); a second
// kernel adds the blocks in a fixed order, so C is the same to the last bit
// from run to run (and graph replay to replay).
constexpr int DOT_BLOCKS = 1184;  // 8 x 148 SMs

// C_ab partial sums over the elements e = (pair i'<j', k') of
//   sum_e gamma^b[e] (Z^a[e] conj(Phi~[e])),  gamma^b = g^b_i' g^b_j' g^b_k',
// Phi~[e] = the source elemental at the sorted (i', j', k') with the sign of
// the sort (0 if k' is i' or j').  A block of 32 nb threads takes tiles of
// 32 nb elements: first every thread forms conj(Phi~) and the nb weights
// gamma^b of one element into shared memory, then warp a runs over the tile
// with a = its warp, one element per lane at a time, keeping the nb complex
// sums C_ab as unevaluated double-floats.
template <int MAXB>
__global__ void __launch_bounds__(32 * MAXB)
dot_z_kernel(const CDF* __restrict__ Z, const CDF* __restrict__ phi_all, const DF* __restrict__ g, int nv, int nb,
             Cx<double>* __restrict__ part_all) {
  __shared__ CDF sphi[32 * MAXB];
  __shared__ DF sgam[MAXB][32 * MAXB];
  const int tile = 32 * nb;
  const int a = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long P2 = comb2(nv);
  const long long work = P2 * nv;
  // momentum qb of the batch: its Z slabs, source elementals and partial sums
  const int qb = blockIdx.y;
  const CDF* phi = phi_all + (long long)qb * comb3(nv);
  Cx<double>* part = part_all + (long long)qb * gridDim.x * nb * nb;
  Z += (long long)qb * nb * work;
  float sr[MAXB], cr[MAXB], si[MAXB], ci[MAXB];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) sr[b] = cr[b] = si[b] = ci[b] = 0.f;
  const CDF* Za = Z + (long long)a * work;
  for (long long e0 = (long long)blockIdx.x * tile; e0 < work; e0 += (long long)gridDim.x * tile) {
    {  // phase 1: one element per thread
      const long long e = e0 + threadIdx.x;
      CDF f = cdf_zero();
      DF gm[MAXB];
#pragma unroll
      for (int b = 0; b < MAXB; ++b) gm[b] = df_make(0.f, 0.f);
      if (e < work) {
        const long long pair = e / nv;
        const int kp = (int)(e - pair * nv);
        int ip, jp;
        pair_unrank(pair, ip, jp);
        if (kp != ip && kp != jp) {
          f = cdf_conj(phi_at(phi, ip, jp, kp, df_make(1.f, 0.f)));
#pragma unroll
          for (int b = 0; b < MAXB; ++b) {
            if (b >= nb) break;
            const DF* gb = g + (long long)b * nv;
            gm[b] = df_mul(df_mul(gb[ip], gb[jp]), gb[kp]);
          }
        }
      }
      sphi[threadIdx.x] = f;
#pragma unroll
      for (int b = 0; b < MAXB; ++b)
        if (b < nb) sgam[b][threadIdx.x] = gm[b];
    }
    __syncthreads();
    // phase 2: warp a over the tile
    for (int i = lane; i < tile; i += 32) {
      const long long e = e0 + i;
      if (e >= work) break;
      const CDF z = ldg_cdf(Za + e);
      const CDF f = sphi[i];
      // u = z f (complex double-float product)
      const DF ur = df_sub(df_mul(z.re, f.re), df_mul(z.im, f.im));
      const DF ui = df_add(df_mul(z.re, f.im), df_mul(z.im, f.re));
#pragma unroll
      for (int b = 0; b < MAXB; ++b) {
        if (b >= nb) break;
        const DF gb = sgam[b][i];
        df_acc_prod(sr[b], cr[b], gb, ur);
        df_acc_prod(si[b], ci[b], gb, ui);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    if (b >= nb) break;
    DF vr = two_sum(sr[b], cr[b]), vi = two_sum(si[b], ci[b]);
    for (int o = 16; o > 0; o >>= 1) {
      vr = df_add(vr, df_make(__shfl_xor_sync(0xffffffffu, vr.hi, o), __shfl_xor_sync(0xffffffffu, vr.lo, o)));
      vi = df_add(vi, df_make(__shfl_xor_sync(0xffffffffu, vi.hi, o), __shfl_xor_sync(0xffffffffu, vi.lo, o)));
    }
    if (lane == 0) {
      Cx<double>& dst = part[((long long)blockIdx.x * nb + a) * nb + b];
      dst.r = df_to_double(vr);
      dst.i = df_to_double(vi);
    }
  }
}

// C[a][b] = 2^scale sum over blocks of part[block][a][b]: one block of 256
// threads per (a, b) and momentum qb = blockIdx.y of the batch, each thread
// summing a fixed stride of the blocks, then a fixed-shape tree, so the
// order of the additions never changes.  The exponents of momentum qb are
// esnk[qb], esrc[qb]; its C block starts cstride_q further on.
__global__ void __launch_bounds__(256)
dot_reduce_kernel(const Cx<double>* __restrict__ part, int nblocks, int nb, const int* __restrict__ etau,
                  const int* __restrict__ esnk, const int* __restrict__ esrc, Cx<double>* __restrict__ C,
                  long long cstride_a, long long cstride_b, long long cstride_q) {
  __shared__ double sr[256], si[256];
  const int ab = blockIdx.x, qb = blockIdx.y;
  part += (long long)qb * nblocks * nb * nb;
  double zr = 0.0, zi = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += 256) {
    const Cx<double> p = part[(long long)k * nb * nb + ab];
    zr += p.r;
    zi += p.i;
  }
  sr[threadIdx.x] = zr;
  si[threadIdx.x] = zi;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sr[threadIdx.x] += sr[threadIdx.x + h];
      si[threadIdx.x] += si[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double scale = ldexp(1.0, 3 * etau[0] + esnk[qb] + esrc[qb]);
    Cx<double>& dst = C[qb * cstride_q + (ab / nb) * cstride_a + (ab % nb) * cstride_b];
    dst.r = sr[0] * scale;
    dst.i = si[0] * scale;
  }
}

// ------------------------------------------------------------------ workspace
struct MixedWs {
  PlaneImg Aa, TT, TcT, G, U, W;  // operand plane images
  int *eAa, *eTT, *eTcT, *eG, *eU, *eW;
  float *nAa, *nG, *mG;
  CDF *V, *Z, *phs, *ph0;
  Cx<double>* part;
  DF* g;
  int *etau, *esnk, *esrc;
  int nvp;  // rows of each b' block of TT: N_v rounded up to 8
};

// Per-timeslice buffers (the tau splits) once; per-momentum buffers for a
// group of pb momenta processed together.
static MixedWs carve_mixed(Arena& ar, const Scheme& sc, int nt, int nv, int np, int nb, int pb) {
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv), T3 = comb3(nv);
  const int npa = 2 * sc.na, npb = 2 * sc.nb;
  const long long bq = (long long)pb * nb;  // (momentum, profile) slabs of a group
  MixedWs w;
  w.nvp = (nv + 7) / 8 * 8;
  const long long n5 = (long long)NSRC * n, r4 = 4LL * w.nvp;
  auto img = [&ar](long long K, long long rows, long long coords, int planes) {
    return tc::plane_img(ar.take<uint16_t>(tc::plane_img_elems(K, rows, coords, planes)), K, rows, coords, planes);
  };
  w.Aa = img(n, n, 12, npa);
  w.TT = img(4 * n, r4, 1, npb);
  w.TcT = img(n5, n, 1, npb);
  w.G = img(n, n2, bq, npb);
  w.U = img(4 * n, n2, 3 * bq, npa);
  w.W = img(n5, P2, bq, npa);
  w.eAa = ar.take<int>(12 * n);
  w.eTT = ar.take<int>(r4);
  w.eTcT = ar.take<int>(n);
  w.eG = ar.take<int>(bq * n2);
  w.eU = ar.take<int>(3 * bq * n2);
  w.eW = ar.take<int>(bq * P2);
  w.nAa = ar.take<float>(12 * n);
  w.nG = ar.take<float>(bq * n2);
  w.mG = ar.take<float>(bq * n);
  w.V = ar.take<CDF>(bq * NPAIR * n3);
  w.part = ar.take<Cx<double>>((long long)pb * DOT_BLOCKS * nb * nb);
  w.Z = ar.take<CDF>(bq * P2 * n);
  w.phs = ar.take<CDF>((long long)pb * T3);
  w.ph0 = ar.take<CDF>((long long)pb * T3);
  w.g = ar.take<DF>((long long)(nt + 1) * nb * n);
  w.etau = ar.take<int>(nt);
  w.esnk = ar.take<int>((long long)nt * np);
  w.esrc = ar.take<int>(np);
  return w;
}

// Momenta processed together: as many as fit a 32 GiB workspace (all of
// them for N_v <= 128; one at a time at N_v = 256, whose correlator alone
// needs ~40 GB).
constexpr size_t MIXED_GROUP_BUDGET = size_t(32) << 30;
static int mixed_group(const Scheme& sc, int nt, int nv, int np, int nb) {
  Arena one, two;
  carve_mixed(one, sc, nt, nv, np, nb, 1);
  carve_mixed(two, sc, nt, nv, np, nb, 2);
  const size_t per = two.used - one.used, base = one.used - per;
  int pb = 1;
  while (pb < np && base + (size_t)(pb + 1) * per <= MIXED_GROUP_BUDGET) ++pb;
  return pb;
}

size_t correlate_mixed_workspace(int mode, int nt, int nv, int np, int nb) {
  const Scheme sc = scheme_of(mode);
  Arena ar;
  carve_mixed(ar, sc, nt, nv, np, nb, mixed_group(sc, nt, nv, np, nb));
  return ar.used + 256;
}

// Mode-contraction GEMM in the kernel variant the context's tuning table
// names for this site (step i, step j, and the T contraction with K = 5 N_v,
// which took the tuning slot of the former source-side contraction):
//   0  one 128 x NT tile per CTA, NT the widest TMEM allows (128, or 80 /
//      64 by padding cost with three accumulator pairs); no overlap of
//      epilogue and MMAs
//   1  persistent CTAs with two accumulator sets (the epilogue of one tile
//      overlaps the MMAs of the next), 128 x 64 (128 x 32 with three pairs)
//   2  step i only: as 1 with the whole-K A tile resident in shared memory
//      across the column tiles of a batch (K <= 128; else variant 1)
//   3  one 128 x 64 tile per CTA
//   4  persistent, 128 x 32 tiles
//   5  persistent with one accumulator set of the widest tile (128, or 80 /
//      64 with three pairs): the MMAs of a tile wait for the previous
//      epilogue, the copy ring fills meanwhile
// NACC is a property of the site, not of the variant: step j (K = 4 N_v) and the T contraction (K = 5 N_v)
// accumulate the 6-product schemes in three pairs (exact cross terms; the
// second-order terms drift with K otherwise), step i (K = N_v) in two.  All variants of a site
// accumulate every element over K in the same order into the same pairs, so
// they give identical results.
enum GemmSite { SITE_STEP_I = 0, SITE_STEP_J = 1, SITE_SOURCE = 2 };
template <bool BF16, int NPLA, int NPLB, int NACC, class Epi>
static int gemm(distil_ctx* ctx, GemmSite site, const char* name, const PlaneImg& A, const PlaneImg& B,
                const tc::GemmCfg& cfg, int batch, const Epi& epi, cudaStream_t s) {
  constexpr int KC = 16;
  constexpr int NKA = 8;  // resident A covers K <= 128
  constexpr int NTP = NACC == 3 ? 32 : 64;    // persistent: two sets of 2 NACC NT columns
  constexpr int NTW = NACC == 3 ? 80 : 128;   // one-tile: 2 NACC NT columns
  const int var = ctx->tune[site];
  if constexpr (NACC == 1) {
    // the second-order pass of a split contraction: two 128-wide sets
    // (2 x 2 x 128 TMEM columns), the epilogue of one tile under the MMAs
    // of the next
    (void)var;
    if (cfg.N > 64)
      return tc::launch_gemm_persistent<128, KC, NPLA, NPLB, tc::max_stages<128, KC, NPLA, NPLB>(), BF16, 1, 2>(
          ctx, name, A, B, cfg, batch, epi, s);
    return tc::launch_gemm_persistent<64, KC, NPLA, NPLB, tc::max_stages<64, KC, NPLA, NPLB>(), BF16, 1, 2>(
        ctx, name, A, B, cfg, batch, epi, s);
  } else {
  if (var == 5 && cfg.N > 64) {
    if constexpr (NACC == 3) {
      const double c80 = ((cfg.N + 79) / 80) * 80 * (1.0 / 80 + 1.0 / 128);
      const double c64 = ((cfg.N + 63) / 64) * 64 * (1.0 / 64 + 1.0 / 128);
      if (c64 < c80)
        return tc::launch_gemm_persistent<64, KC, NPLA, NPLB, tc::max_stages<64, KC, NPLA, NPLB>(), BF16, NACC, 1>(
            ctx, name, A, B, cfg, batch, epi, s);
    }
    return tc::launch_gemm_persistent<NTW, KC, NPLA, NPLB, tc::max_stages<NTW, KC, NPLA, NPLB>(), BF16, NACC, 1>(
        ctx, name, A, B, cfg, batch, epi, s);
  }
  if constexpr (NACC == 2) {
    if (var == 2 && cfg.K <= NKA * KC && cfg.N > 32)
      return tc::launch_gemm_ares<64, KC, NPLA, NPLB, NKA, BF16, NACC>(ctx, name, A, B, cfg, batch, epi, s);
    if (var == 4)  // persistent, narrow tiles
      return tc::launch_gemm_persistent<32, KC, NPLA, NPLB, tc::max_stages<32, KC, NPLA, NPLB>(), BF16, NACC>(
          ctx, name, A, B, cfg, batch, epi, s);
  }
  if (var == 1 || var == 2 || var == 4) {
    if (cfg.N > 32)
      return tc::launch_gemm_persistent<NTP, KC, NPLA, NPLB, tc::max_stages<NTP, KC, NPLA, NPLB>(), BF16, NACC>(
          ctx, name, A, B, cfg, batch, epi, s);
    return tc::launch_gemm_persistent<32, KC, NPLA, NPLB, tc::max_stages<32, KC, NPLA, NPLB>(), BF16, NACC>(
        ctx, name, A, B, cfg, batch, epi, s);
  }
  if (cfg.N > 64 && var == 0) {
    if constexpr (NACC == 3) {
      // 80-wide tiles read A once per 80 columns, 64-wide ones waste no
      // padding when N is a multiple of 64: shared-memory reads per output
      // ~ padded columns x (1/NT + 1/128)
      const double c80 = ((cfg.N + 79) / 80) * 80 * (1.0 / 80 + 1.0 / 128);
      const double c64 = ((cfg.N + 63) / 64) * 64 * (1.0 / 64 + 1.0 / 128);
      if (c64 < c80)
        return tc::launch_gemm<64, KC, NPLA, NPLB, tc::max_stages<64, KC, NPLA, NPLB>(), BF16, NACC>(
            ctx, name, A, B, cfg, batch, epi, s);
    }
    return tc::launch_gemm<NTW, KC, NPLA, NPLB, tc::max_stages<NTW, KC, NPLA, NPLB>(), BF16, NACC>(
        ctx, name, A, B, cfg, batch, epi, s);
  }
  // variant 3, and narrow N: one-tile, 64 (or 32) wide
  if (cfg.N > 32)
    return tc::launch_gemm<64, KC, NPLA, NPLB, tc::max_stages<64, KC, NPLA, NPLB>(), BF16, NACC>(ctx, name, A, B, cfg,
                                                                                                batch, epi, s);
  return tc::launch_gemm<32, KC, NPLA, NPLB, tc::max_stages<32, KC, NPLA, NPLB>(), BF16, NACC>(ctx, name, A, B, cfg,
                                                                                              batch, epi, s);
  }
}

// A long contraction of the 3 x 4 piece schemes in two passes over the same
// plane images, so that no pass needs more than two accumulator pairs and
// the MMAs run 128 wide (three pairs fit TMEM only 80 wide, and 80-wide
// MMAs take ~1.3x the time per column):
//   pass A  the leading two pieces of each side: hi*hi | hi*mid + mid*hi,
//           both pairs exact integer sums, stored by epi as D0 + D1;
//   pass B  the second-order terms hi*lo, mid*mid', lo*hi in one pair,
//           added into the stored values in double-float by epi_add.
// A holds the pieces hi, mid, lo (pass A reads its first four planes), B
// the pieces in the order mid', lo, hi, mid, so that pass A reads B's last
// four planes and pass B its first six: no pass copies a plane it does not
// use.  The classes accumulate exactly as with three pairs; D1 and D2 now
// meet in double-float instead of FP32.
template <bool BF16, class EpiS, class EpiA>
static int contract_two_pass(distil_ctx* ctx, GemmSite site, const char* name, const char* name_2nd,
                             const PlaneImg& A, const PlaneImg& B, tc::GemmCfg cfg, int batch, const EpiS& epi,
                             const EpiA& epi_add, cudaStream_t s) {
  using PA = tc::SchemeProducts<4, 4, 2>;
  cfg.nprod = PA::n;
  for (int p = 0; p < PA::n; ++p) {
    cfg.pa[p] = PA::pa[p];
    cfg.pb[p] = PA::pb[p];
  }
  DISTIL_TRY((gemm<BF16, 4, 4, 2>(ctx, site, name, tc::plane_view(A, 0, 4), tc::plane_view(B, 4, 4), cfg, batch, epi, s)));
  using PB = tc::SchemeProducts<6, 6, 1>;
  cfg.nprod = PB::n;
  for (int p = 0; p < PB::n; ++p) {
    cfg.pa[p] = PB::pa[p];
    cfg.pb[p] = PB::pb[p];
  }
  return gemm<BF16, 6, 6, 1>(ctx, site, name_2nd, A, tc::plane_view(B, 0, 6), cfg, batch, epi_add, s);
}

static inline unsigned nblk(long long work, int bs = 256) { return (unsigned)((work + bs - 1) / bs); }

// The tau splits of timeslice t (shared by every momentum).
template <bool BF16, bool FIXED, int NA, int NB>
static int split_tau_t(distil_ctx* ctx, const Scheme& sch, const float2* tau, const int* etau, int nv,
                       const MixedWs& w, cudaStream_t s) {
  const long long n = nv;
  const int H = sch.H;
  DISTIL_TRY((split_rows<BF16, FIXED, NA>(ctx, "split_tau", AaSrc{tau, etau, nv}, 12 * n, w.Aa, H, w.eAa, s, w.nAa)));
  // the B operands of the two-pass contractions (four pieces) in the piece
  // order mid', lo, hi, mid (contract_two_pass)
  constexpr int ROT = NB == 4 ? 2 : 0;
  DISTIL_TRY((split_rows<BF16, FIXED, NB, TTSrc, ROT>(ctx, "split_tau", TTSrc{tau, etau, nv, w.nvp}, 4LL * w.nvp, w.TT, H, w.eTT, s)));
  DISTIL_TRY((split_rows<BF16, FIXED, NB, TcTSrc, ROT>(ctx, "split_tau", TcTSrc{TcSrc{tau, etau, nv}}, n, w.TcT, H, w.eTcT, s)));
  return DISTIL_OK;
}

// C_ab(t) of a group of pb momenta q0 .. q0 + pb - 1 at one timeslice, the
// tau splits of the timeslice already in w: phs_c128 / ph0_c128 point at the
// group's first sink / source elementals (stride T3), esnk / esrc at its
// first exponents, Cout at C[q0][0][0][t] (momentum stride cs_q).
template <bool BF16, bool FIXED, int NA, int NB>
static int run_group_mixed(distil_ctx* ctx, const Scheme& sch, int pb, const double2* phs_c128,
                           const double2* ph0_c128, const DF* g_snk, const DF* g_src, const int* etau,
                           const int* esnk, const int* esrc, int nv, int nb, const MixedWs& w, Cx<double>* Cout,
                           long long cs_a, long long cs_b, long long cs_q, cudaStream_t s) {
  constexpr int NPLA = 2 * NA, NPLB = 2 * NB;
  const long long n = nv, n2 = n * n, n3 = n2 * n, P2 = comb2(nv), T3 = comb3(nv);
  const long long bq = (long long)pb * nb;  // (momentum, profile) slabs
  using P16 = typename tc::Piece<BF16>::T;
  {
    Launch L(ctx, "normalise", s);
    c128_to_cdf_kernel<<<dim3(nblk(T3), pb), 256, 0, s>>>(phs_c128, T3, T3, esnk, w.phs);
    c128_to_cdf_kernel<<<dim3(nblk(T3), pb), 256, 0, s>>>(ph0_c128, T3, T3, esrc, w.ph0);
  }
  // ---- sink operand (rows (momentum, profile, k, j), per-row exponents)
  const int H = sch.H;
  DISTIL_TRY((split_rows<BF16, FIXED, NB>(ctx, "split_sink", GSrc{w.phs, g_snk, nv, nb, T3}, bq * n2, w.G, H, w.eG, s, w.nG)));
  {
    Launch L(ctx, "u_exponent", s);
    g_rowmax_kernel<<<nblk(32LL * bq * n), 256, 0, s>>>(w.nG, nv, (int)bq, w.mG);
    u_exponent_kernel<<<nblk(3 * bq * n2), 256, 0, s>>>(w.nAa, w.mG, nv, (int)bq, w.eU);
  }
  DISTIL_LAUNCH_CHECK();

  tc::GemmCfg cfg{};
  fill_products(cfg, sch);
  cfg.err = ctx->d_error;

  // ---- step i: batch (momentum, a, a'beta) = pb x nb x 12, output split into U pieces
  {
    cfg.M = nv; cfg.N = (int)n2; cfg.K = nv;
    cfg.a = tc::OpMap{1, 12, 1, 0, 0, nv, w.eAa};
    cfg.b = tc::OpMap{12, (int)bq, 1, 0, 0, (int)n2, w.eG};
    EpiSplitU<BF16, FIXED, NA> epi{{}, w.U, w.eU, nv, H};
    cfg.order = 1;  // the 2 x 12 tiles that read one G tile run back to back
    DISTIL_TRY((gemm<BF16, NPLA, NPLB, 2>(ctx, SITE_STEP_I, "tc_gemm_step_i", w.Aa, w.G, cfg, (int)bq * 12, epi, s)));
    cfg.order = 0;
  }
  // ---- step j: per a' (rows b' > a'), batch (momentum, a); V[qa][slot][j'][(i',k)]
  const int slotbase[3] = {0, 3, 5};
  for (int ap = 0; ap < 3; ++ap) {
    // columns (b', j') over the b' blocks of nvp rows; j' >= N_v is padding
    const int nvp = w.nvp;
    cfg.M = (int)n2; cfg.N = (3 - ap) * nvp; cfg.K = 4 * nv;
    cfg.a = tc::OpMap{1, (int)bq, 3, ap, 0, (int)n2, w.eU};
    cfg.b = tc::OpMap{1, 1, 0, 0, (ap + 1) * nvp, 4 * nvp, w.eTT};
    EpiStoreCDF epi;
    epi.out = w.V + (long long)slotbase[ap] * n3;
    epi.b_lo = 1; epi.sb_hi = NPAIR * n3; epi.sb_lo = 0;
    epi.sr = 1; epi.cm = ColMap{n2, nvp, n3, nv}; epi.N = (3 - ap) * nvp;
    if constexpr (NPLA == 6) {
      const EpiAddCDF add{{}, epi.out, epi.sb_hi, epi.sb_lo, epi.b_lo, epi.sr, epi.cm, epi.N};
      DISTIL_TRY((contract_two_pass<BF16>(ctx, SITE_STEP_J, "tc_gemm_step_j", "tc_gemm_step_j_2nd", w.U, w.TT, cfg, (int)bq, epi, add, s)));
    } else {
      DISTIL_TRY((gemm<BF16, NPLA, NPLB, 2>(ctx, SITE_STEP_J, "tc_gemm_step_j", w.U, w.TT, cfg, (int)bq, epi, s)));
    }
  }
  // ---- W: the source-weighted antisymmetric parts of V, split (rows (momentum, a, pair), K = (c, k))
  {
    Launch L(ctx, "split_w", s);
    const unsigned rows = (unsigned)(bq * P2);
    if (nv <= 256)
      split_w_kernel<BF16, FIXED, NA, 1><<<rows, 256, 0, s>>>(w.V, nv, P2, H, w.W, w.eW);
    else if (nv <= 512)
      split_w_kernel<BF16, FIXED, NA, 2><<<rows, 256, 0, s>>>(w.V, nv, P2, H, w.W, w.eW);
    else
      split_w_kernel<BF16, FIXED, NA, 4><<<rows, 256, 0, s>>>(w.V, nv, P2, H, w.W, w.eW);
  }
  DISTIL_LAUNCH_CHECK();
  // ---- T contraction: Z[qa][pair][k'] = sum_(c,k) W[qa][pair][(c,k)] T^c[k][k'] (K = 5 N_v)
  {
    cfg.M = (int)P2; cfg.N = nv; cfg.K = NSRC * nv;
    cfg.a = tc::OpMap{1, (int)bq, 1, 0, 0, (int)P2, w.eW};
    cfg.b = tc::OpMap{1, 1, 0, 0, 0, nv, w.eTcT};
    EpiStoreCDF epi;
    epi.out = w.Z;
    epi.b_lo = 1; epi.sb_hi = P2 * n; epi.sb_lo = 0;
    epi.sr = n; epi.cm = ColMap{1, 0, 0, 0}; epi.N = nv;
    if constexpr (NPLA == 6) {
      const EpiAddCDF add{{}, epi.out, epi.sb_hi, epi.sb_lo, epi.b_lo, epi.sr, epi.cm, epi.N};
      DISTIL_TRY((contract_two_pass<BF16>(ctx, SITE_SOURCE, "tc_gemm_tcontract", "tc_gemm_tcontract_2nd", w.W, w.TcT, cfg, (int)bq, epi, add, s)));
    } else {
      DISTIL_TRY((gemm<BF16, NPLA, NPLB, 2>(ctx, SITE_SOURCE, "tc_gemm_tcontract", w.W, w.TcT, cfg, (int)bq, epi, s)));
    }
  }
  // ---- dot, then the fixed-order reduction into C (momentum on grid y)
  {
    const long long work = P2 * n;
    const long long tile = 32LL * nb;
    unsigned gx = (unsigned)((work + tile - 1) / tile);
    if (gx > (unsigned)DOT_BLOCKS) gx = DOT_BLOCKS;
    Launch L(ctx, "dot", s);
    if (nb <= 8)
      dot_z_kernel<8><<<dim3(gx, pb), 32 * nb, 0, s>>>(w.Z, w.ph0, g_src, nv, nb, w.part);
    else
      dot_z_kernel<16><<<dim3(gx, pb), 32 * nb, 0, s>>>(w.Z, w.ph0, g_src, nv, nb, w.part);
    dot_reduce_kernel<<<dim3(nb * nb, pb), 256, 0, s>>>(w.part, (int)gx, nb, etau, esnk, esrc, Cout, cs_a, cs_b, cs_q);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

template <bool BF16, bool FIXED, int NA, int NB>
static int correlate_mixed_t(distil_ctx* ctx, const Scheme& sch, const void* phi_snk, const void* phi_src,
                             const void* tau, int nt, int nv, int np, int pb, int prof_per_t, int nb, const DF* g_src,
                             const MixedWs& w, Cx<double>* Cd, int c_nt, int c_t0, cudaStream_t s) {
  const long long T3 = comb3(nv), n4 = 4LL * nv;
  for (int t = 0; t < nt; ++t) {
    const DF* g_snk = w.g + (prof_per_t ? (long long)t * nb * nv : 0);
    const float2* ta = (const float2*)tau + (long long)t * n4 * n4;
    DISTIL_TRY((split_tau_t<BF16, FIXED, NA, NB>(ctx, sch, ta, w.etau + t, nv, w, s)));
    for (int q0 = 0; q0 < np; q0 += pb) {
      const int g = np - q0 < pb ? np - q0 : pb;
      const double2* phs = (const double2*)phi_snk + ((long long)t * np + q0) * T3;
      const double2* ph0 = (const double2*)phi_src + (long long)q0 * T3;
      Cx<double>* Cq = Cd + (long long)q0 * nb * nb * c_nt + c_t0 + t;
      DISTIL_TRY((run_group_mixed<BF16, FIXED, NA, NB>(ctx, sch, g, phs, ph0, g_snk, g_src, w.etau + t,
                                                      w.esnk + (long long)t * np + q0, w.esrc + q0, nv, nb, w, Cq,
                                                      (long long)nb * c_nt, c_nt, (long long)nb * nb * c_nt, s)));
    }
  }
  return DISTIL_OK;
}

int mixed_mode_built(int mode) { return is_mixed(mode) ? 1 : 0; }

int correlate_mixed(distil_ctx* ctx, int mode, const void* phi_snk, const void* phi_src, const void* tau, int nt,
                    int nv, int np, const double* prof_snk, const double* prof_src, int prof_per_t, int nb, void* C,
                    int c_nt, int c_t0, void* ws, size_t ws_bytes, cudaStream_t s) {
  DISTIL_TRY(zero_c_columns(C, (long long)np * nb * nb, c_nt, c_t0, nt, s));
  if (nv < 3) return DISTIL_OK;
  const Scheme sch = scheme_of(mode);
  const int pb = mixed_group(sch, nt, nv, np, nb);
  Arena ar(ws, ws_bytes);
  MixedWs w = carve_mixed(ar, sch, nt, nv, np, nb, pb);
  if (!ar.fits()) {
    set_error("correlate: workspace too small");
    return DISTIL_ENOMEM;
  }
  const long long T3 = comb3(nv), n4 = 4LL * nv;
  const long long nprof = (prof_per_t ? (long long)nt : 1) * nb * nv;
  DF* g_src = w.g + (long long)nt * nb * nv;  // the source profiles follow the sink blocks
  {
    Launch L(ctx, "normalise", s);
    // exponents: every array spread over up to 64 blocks
    const unsigned bt = (unsigned)std::min<long long>(64, (n4 * n4 + 8191) / 8192);
    const unsigned bp = (unsigned)std::min<long long>(64, (T3 + 8191) / 8192);
    exp_init_kernel<<<nblk(nt), 256, 0, s>>>(w.etau, nt);
    exp_init_kernel<<<nblk((long long)nt * np), 256, 0, s>>>(w.esnk, nt * np);
    exp_init_kernel<<<nblk(np), 256, 0, s>>>(w.esrc, np);
    c64_exp_kernel<<<dim3(bt, nt), 256, 0, s>>>((const float2*)tau, n4 * n4, w.etau);
    c128_exp_kernel<<<dim3(bp, nt * np), 256, 0, s>>>((const double2*)phi_snk, T3, w.esnk);
    c128_exp_kernel<<<dim3(bp, np), 256, 0, s>>>((const double2*)phi_src, T3, w.esrc);
    prof_to_df_kernel<<<nblk(nprof), 256, 0, s>>>(prof_snk, nprof, w.g);
    prof_to_df_kernel<<<nblk((long long)nb * nv), 256, 0, s>>>(prof_src, (long long)nb * nv, g_src);
  }
  DISTIL_LAUNCH_CHECK();
  DISTIL_TRY(img_zero_kpad(ctx, w.U, s));  // the step-i epilogue writes K = 4 N_v elements only
  Cx<double>* Cd = reinterpret_cast<Cx<double>*>(C);
  if (mode == DISTIL_MIXED_FP16X6)
    return correlate_mixed_t<false, true, 3, 4>(ctx, sch, phi_snk, phi_src, tau, nt, nv, np, pb, prof_per_t, nb, g_src,
                                                w, Cd, c_nt, c_t0, s);
  if (mode == DISTIL_MIXED_BF16X6)
    return correlate_mixed_t<true, true, 3, 4>(ctx, sch, phi_snk, phi_src, tau, nt, nv, np, pb, prof_per_t, nb, g_src,
                                               w, Cd, c_nt, c_t0, s);
  if (mode == DISTIL_MIXED_BF16X3)
    return correlate_mixed_t<true, true, 2, 2>(ctx, sch, phi_snk, phi_src, tau, nt, nv, np, pb, prof_per_t, nb, g_src,
                                               w, Cd, c_nt, c_t0, s);
  return correlate_mixed_t<false, false, 2, 2>(ctx, sch, phi_snk, phi_src, tau, nt, nv, np, pb, prof_per_t, nb, g_src,
                                               w, Cd, c_nt, c_t0, s);
}

}  // namespace distil
