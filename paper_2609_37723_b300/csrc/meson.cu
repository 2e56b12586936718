// One-meson operators with distillation profiles (paper Sec. 2.3, "Improved
// charmonium operators") on tcgen05 tensor cores:
//
//  elementals  Phi^d[p]_ij = sum_x exp(-i p.x) v_i(x)^dagger (D_d v_j)(x),
//              d = 0..6 for 1, nabla_x,y,z, BB_x,y,z: nabla_k the symmetric
//              covariant difference 1/2 [U_k(x) f(x+k) - U_k(x-k)^dagger
//              f(x-k)], BB_i = nabla_j nabla_k - nabla_k nabla_j ((i,j,k)
//              cyclic);
//  correlate   C_ab(p, t) = -Tr[Phi_a(t) tau(t) Phibar_b(0) g5 tau(t)^dagger g5]
//              for the 3 Gamma x N_B profile operators a = 7 type + sigma
//              (type 0: gamma_4 gamma_5, 1: gamma_4 gamma_5 gamma_k nabla_k,
//              2: gamma_k BB_k);
//  prune       the left singular vectors U_n of C(t_p) for its n largest
//              singular values and Ct(t) = U_n^dagger C(t) U_n.
//
// Elementals, per batch of timeslices: the three nabla_k v fields and then the
// three BB_i v fields are formed once in double-float (exact FP32 products
// summed by compensated dot products); then K = (site, colour) runs in chunks
// of MS_KC values: the A operand rows (d, j) are v or the stored displaced
// fields; the B operand rows (p, i) are
// exp(-i p.x) conj(v_i); the tensor cores accumulate each chunk and the
// epilogue adds it into a double-float Phi_acc[(d, j)][(p, i)].
//
// Correlator, per sink timeslice and momentum, with the spin-major
// 4 N_v x 4 N_v matrices of the operators (every Gamma is a signed
// permutation, so the operand writers form their entries from the
// elementals, the profiles and a phase table):
//   Q_b = Phibar_b tau~,  tau~ = g5 tau^dagger g5      (GEMM 1, stored Q_b^T)
//   X_b = tau Q_b                                      (GEMM 2)
//   C_ab = -sum_c sum_alpha s_c(alpha) sum_ij g_i g_j Phi^(d_c)_ij X_b[(pi_c(alpha), j)][(alpha, i)]
// the last as a CUDA-core reduction in double-float.  The source operand of
// GEMM 1 does not depend on t and is split once per momentum.
#include <math.h>

#include <complex>

#include "df.cuh"
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

using tc::PlaneImg;

constexpr int MS_NDISP = 7;
constexpr int MS_KC = 4032;  // K chunk of the elementals: whole sites, whole K blocks
static_assert(MS_KC % 3 == 0 && MS_KC % 16 == 0, "chunks of whole sites and K blocks");
constexpr int MS_MAX_MOM = 16;
constexpr int MS_MAX_NB = 10;  // 3 N_B <= 30 operators: one warp lane per row in the SVD
constexpr int MS_RED_CHUNKS = 8;  // i chunks of the correlator reduction
// Norm caps (split writers: the scaled slices of a capped row have 2-norm
// <= 2^bits) on the operand rows that can sum coherently against rows of
// the other operand, whose leading-slice sums must stay below 2^24 to add
// exactly: in the elementals v_j (d = 0) against exp(-i p.x) conj(v_i) at
// p = 0 (sum_x |v_i|^2 = 1 on the diagonal); in GEMM 2 the type-0 source
// rows of Q (Phibar ~ identity in mode space, so Q ~ g5 tau^dagger g5)
// against the tau rows.  2^11 x 2^12 keeps those sums below 2^23.  Rows that
// sum with random signs keep their max-based exponents (and their bits):
// capping every row cost up to five bits of GEMM 2.
constexpr int MS_CAP_A = 11, MS_CAP_B = 12;

// ------------------------------------------------------------ spin tables
// Gamma[alpha][perm[alpha]] = phase[alpha] (a signed permutation, phases in
// {+-1, +-i}) for the sink Gammas of the seven displacements, their source
// partners gamma_4 Gamma^dagger gamma_4, and gamma_5.
struct SpinTab {
  int perm[MS_NDISP][4];
  int ph[MS_NDISP][4];  // phase i^ph
};
struct SpinTabs {
  SpinTab snk, src;
  int g5perm[4];
  int g5ph[4];
};

namespace {
using z4 = std::complex<double>;
struct M4 {
  z4 a[4][4];
};
M4 mul(const M4& x, const M4& y) {
  M4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) r.a[i][j] += x.a[i][k] * y.a[k][j];
  return r;
}
M4 dag(const M4& x) {
  M4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r.a[i][j] = std::conj(x.a[j][i]);
  return r;
}
// Euclidean Dirac-Pauli gammas: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
// gamma_4 = diag(1, 1, -1, -1)
M4 gamma(int mu) {
  const z4 I(0, 1);
  z4 s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  M4 r{};
  if (mu == 3) {
    r.a[0][0] = r.a[1][1] = 1;
    r.a[2][2] = r.a[3][3] = -1;
    return r;
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      r.a[i][2 + j] = -I * s[mu][i][j];
      r.a[2 + i][j] = I * s[mu][i][j];
    }
  return r;
}
bool to_perm(const M4& g, int* perm, int* ph) {
  for (int i = 0; i < 4; ++i) {
    int n = 0;
    for (int j = 0; j < 4; ++j) {
      const z4 v = g.a[i][j];
      if (std::abs(v) < 1e-12) continue;
      ++n;
      perm[i] = j;
      if (std::abs(v - z4(1, 0)) < 1e-12) ph[i] = 0;
      else if (std::abs(v - z4(0, 1)) < 1e-12) ph[i] = 1;
      else if (std::abs(v - z4(-1, 0)) < 1e-12) ph[i] = 2;
      else if (std::abs(v - z4(0, -1)) < 1e-12) ph[i] = 3;
      else return false;
    }
    if (n != 1) return false;
  }
  return true;
}
}  // namespace

static bool spin_tables(SpinTabs& t) {
  const M4 g4 = gamma(3);
  const M4 g5 = mul(mul(mul(gamma(0), gamma(1)), gamma(2)), g4);
  const M4 g45 = mul(g4, g5);
  bool ok = to_perm(g5, t.g5perm, t.g5ph);
  for (int a = 0; ok && a < 4; ++a) ok = t.g5perm[t.g5perm[a]] == a;  // the backward propagator assumes it
  for (int d = 0; d < MS_NDISP; ++d) {
    const M4 G = d == 0 ? g45 : d <= 3 ? mul(g45, gamma(d - 1)) : gamma(d - 4);
    ok = ok && to_perm(G, t.snk.perm[d], t.snk.ph[d]);
    ok = ok && to_perm(mul(mul(g4, dag(G)), g4), t.src.perm[d], t.src.ph[d]);
  }
  return ok;
}

// --------------------------------------------------------- device helpers

// Compensated dot product (Ogita, Rump and Oishi's Dot2): exact products
// (TwoProduct), leading parts summed by TwoSum, every rounding term added
// into c; the result is as accurate as a sum in twice FP32's precision.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const DF t = two_sum(s, p);
    s = t.hi;
    c += t.lo + e;
  }
  __device__ __forceinline__ void add_df(float a, DF b) {
    add(a, b.hi);
    c = __fmaf_rn(a, b.lo, c);
  }
  __device__ __forceinline__ void add_dd(DF a, DF b) {
    add(a.hi, b.hi);
    c = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, c));
  }
  __device__ __forceinline__ DF get() const { return two_sum(s, c); }
};

__device__ __forceinline__ DF df_half(DF a) { return df_make(a.hi * 0.5f, a.lo * 0.5f); }

// i^ph z (exact)
__device__ __forceinline__ CDF cdf_iph(CDF z, int ph) {
  switch (ph & 3) {
    case 0: return z;
    case 1: return cdf_make(df_neg(z.im), z.re);
    case 2: return cdf_make(df_neg(z.re), df_neg(z.im));
    default: return cdf_make(z.im, df_neg(z.re));
  }
}

// Sites s + e_k and s - e_k on the periodic L^3 lattice, s = x + L (y + L z),
// from the coordinates c[3] = (x, y, z) of s.
__device__ __forceinline__ void neighbours(int s, const int (&c)[3], int L, int k, int& sp, int& sm) {
  const int stride = k == 0 ? 1 : k == 1 ? L : L * L;
  sp = c[k] == L - 1 ? s - (L - 1) * stride : s + stride;
  sm = c[k] == 0 ? s + (L - 1) * stride : s - stride;
}

// (nabla_k f)(s)_a accumulated (times sg) into re, im:
//   sum_b U_k(s)_ab f(s+k)_b - conj(U_k(s-k)_ba) f(s-k)_b   (the 1/2 by the caller)
// for an FP32 field f[V3][3] (links Uk[V3][3][3]).
__device__ __forceinline__ void nabla_acc_f(Dot2& re, Dot2& im, float sg, const float2* __restrict__ Uk,
                                            const float2* __restrict__ f, int sp, int s, int sm, int a) {
  const float2* u = Uk + (long long)s * 9 + a * 3;  // row a of U_k(s)
  const float2* w = Uk + (long long)sm * 9 + a;     // column a of U_k(s-k)
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float2 U = u[b], F = f[(long long)sp * 3 + b];
    re.add(sg * U.x, F.x);
    re.add(-sg * U.y, F.y);
    im.add(sg * U.x, F.y);
    im.add(sg * U.y, F.x);
    const float2 W = w[3 * b], G = f[(long long)sm * 3 + b];
    // - conj(W) G = -(W.x G.x + W.y G.y) - i (W.x G.y - W.y G.x)
    re.add(-sg * W.x, G.x);
    re.add(-sg * W.y, G.y);
    im.add(-sg * W.x, G.y);
    im.add(sg * W.y, G.x);
  }
}
// the same for a double-float field F[V3][3]
__device__ __forceinline__ void nabla_acc_df(Dot2& re, Dot2& im, float sg, const float2* __restrict__ Uk,
                                             const CDF* __restrict__ F, int sp, int s, int sm, int a) {
  const float2* u = Uk + (long long)s * 9 + a * 3;
  const float2* w = Uk + (long long)sm * 9 + a;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float2 U = u[b];
    const CDF X = ld_cdf(F + (long long)sp * 3 + b);
    re.add_df(sg * U.x, X.re);
    re.add_df(-sg * U.y, X.im);
    im.add_df(sg * U.x, X.im);
    im.add_df(sg * U.y, X.re);
    const float2 W = w[3 * b];
    const CDF Y = ld_cdf(F + (long long)sm * 3 + b);
    re.add_df(-sg * W.x, Y.re);
    re.add_df(-sg * W.y, Y.im);
    im.add_df(-sg * W.x, Y.im);
    im.add_df(sg * W.y, Y.re);
  }
}

// nabla fields N[u][k][j][s][a] = (nabla_k v_j)(s)_a (fields 0..2 of the
// batch's displaced-field buffer, [u][6][nv][V3][3]) for the timeslices of a
// batch: one thread per (u, k, j, s), three colours.
__global__ void __launch_bounds__(256) meson_nabla_kernel(const float2* __restrict__ v, const float2* __restrict__ U,
                                                          int L, int nv, int tb, CDF* __restrict__ out) {
  const long long V3 = (long long)L * L * L;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)tb * 3 * nv * V3;
  if (idx >= total) return;
  const int s = (int)(idx % V3);
  const long long r = idx / V3;  // (u, k, j)
  const int j = (int)(r % nv);
  const int k = (int)((r / nv) % 3);
  const long long u = r / (3LL * nv);
  const float2* f = v + (u * nv + j) * V3 * 3;
  const float2* Uk = U + (u * 3 + k) * V3 * 9;
  const int c[3] = {s % L, (s / L) % L, s / (L * L)};
  int sp, sm;
  neighbours(s, c, L, k, sp, sm);
  CDF* o = out + ((u * 6 + k) * nv + j) * V3 * 3 + (long long)s * 3;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Dot2 re, im;
    nabla_acc_f(re, im, 1.f, Uk, f, sp, s, sm, a);
    o[a] = cdf_make(df_half(re.get()), df_half(im.get()));
  }
}

// BB fields (fields 3..5 of the buffer): BB_i v_j = nabla_j'(N_k') -
// nabla_k'(N_j') for (i, j', k') cyclic, from the nabla fields N_k = fields
// 0..2.  One thread per (u, j, s), all three i and colours: the outer
// derivative in direction m enters BB_(m+2) with N_(m+1) and BB_(m+1) with
// -N_(m+2), so each link pair U_m(s), U_m(s - m) serves two fields and each
// nabla field is read once (a thread per (u, i, j, s) ran no faster: it
// halved the registers but doubled the field reads and hit the L2 tag rate).
__global__ void __launch_bounds__(128) meson_bb_kernel(const float2* __restrict__ U, int L, int nv, int tb,
                                                       CDF* __restrict__ N) {
  const long long V3 = (long long)L * L * L;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)tb * nv * V3) return;
  const int s = (int)(idx % V3);
  const long long r = idx / V3;
  const int j = (int)(r % nv);
  const long long u = r / nv;
  const int c[3] = {s % L, (s / L) % L, s / (L * L)};
  const long long fs = (long long)nv * V3 * 3;  // stride of one field
  CDF* Nu = N + u * 6 * fs + (long long)j * V3 * 3;
  Dot2 re[3][3], im[3][3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    int sp, sm;
    neighbours(s, c, L, m, sp, sm);
    const float2* Um = U + (u * 3 + m) * V3 * 9;
    const int i_plus = (m + 2) % 3, i_minus = (m + 1) % 3;
    const CDF* f_plus = Nu + ((m + 1) % 3) * fs;
    const CDF* f_minus = Nu + ((m + 2) % 3) * fs;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      nabla_acc_df(re[i_plus][a], im[i_plus][a], 1.f, Um, f_plus, sp, s, sm, a);
      nabla_acc_df(re[i_minus][a], im[i_minus][a], -1.f, Um, f_minus, sp, s, sm, a);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    CDF* o = Nu + (3 + i) * fs + (long long)s * 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = cdf_make(df_half(re[i][a].get()), df_half(im[i][a].get()));
  }
}

__global__ void meson_phase_table_kernel(int L, CDF* tab) {
  const int m = threadIdx.x + blockIdx.x * blockDim.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)L, &s, &c);
  tab[m] = cdf_make(df_from_double(c), df_from_double(-s));  // exp(-2 pi i m / L)
}

struct MsMom {
  int np, L;
  int mom[MS_MAX_MOM][3];
};

// A operand of the elementals: (D_d v_j)(x)_a at K = 3 x + a from K0: v_j
// itself (d = 0) or the stored displaced field d - 1 (nabla_x,y,z, BB_x,y,z)
struct DispRow {
  const float2* v;  // v_j [V3][3]            (d = 0)
  const CDF* f;     // field d - 1 of v_j     (d >= 1)
  int d, K0;
  __device__ __forceinline__ CDF operator()(int kk) const {
    const int K = K0 + kk;
    if (d == 0) {
      const float2 x = v[K];
      return cdf_make(df_make(x.x, 0.f), df_make(x.y, 0.f));
    }
    return ld_cdf(f + K);
  }
  __device__ __forceinline__ float2 approx(int kk) const {
    const CDF z = (*this)(kk);
    return make_float2(z.re.hi, z.im.hi);
  }
};
struct DispSrc {  // rows u (7 nv) + d nv + j
  const float2* v;
  const CDF* N;  // [tb][6][nv][V3][3]
  int nv, K0;
  long long V3;
  __device__ __forceinline__ DispRow row(long long r) const {
    const long long per = (long long)MS_NDISP * nv;
    const long long u = r / per;
    const int rr = (int)(r - u * per);
    const int d = rr / nv, j = rr - d * nv;
    DispRow w{};
    w.d = d;
    w.K0 = K0;
    w.v = v + (u * nv + j) * V3 * 3;
    if (d >= 1) w.f = N + ((u * 6 + (d - 1)) * nv + j) * V3 * 3;
    return w;
  }
  __device__ __forceinline__ CDF operator()(long long r, int kk) const { return row(r)(kk); }
  __device__ __forceinline__ float2 approx(long long r, int kk) const { return row(r).approx(kk); }
  __device__ __forceinline__ int norm_bits(long long r) const {
    return (int)((r % ((long long)MS_NDISP * nv)) / nv) == 0 ? MS_CAP_A : 0;  // d = 0: v_j itself
  }
};

// B operand of the elementals: exp(-i p_q.x) conj(v_i^a(x)) at K = 3 x + a
struct PhConjRow {
  const float2* vi;
  const CDF* tab;
  int m0, m1, m2, L, K0;
  __device__ __forceinline__ CDF operator()(int kk) const {
    const int K = K0 + kk;
    const int x = K / 3;
    const int xy = x / L, xs = x - xy * L, zs = xy / L, ys = xy - zs * L;
    const CDF e = tab[(m0 * xs + m1 * ys + m2 * zs) % L];
    const float2 u = vi[K];
    // (e.re + i e.im)(u.x - i u.y)
    return cdf_make(df_add(df_mul_f(e.re, u.x), df_mul_f(e.im, u.y)),
                    df_sub(df_mul_f(e.im, u.x), df_mul_f(e.re, u.y)));
  }
  __device__ __forceinline__ float2 approx(int kk) const {
    const CDF z = (*this)(kk);
    return make_float2(z.re.hi, z.im.hi);
  }
};
struct PhConjSrc {  // rows u R + q nv + i
  const float2* v;
  const CDF* tab;
  MsMom m;
  int nv, K0;
  long long V3;
  __device__ __forceinline__ PhConjRow row(long long r) const {
    const long long R = (long long)m.np * nv;
    const long long u = r / R;
    const int rr = (int)(r - u * R);
    const int q = rr / nv, i = rr - q * nv;
    return PhConjRow{v + (u * nv + i) * V3 * 3, tab, m.mom[q][0], m.mom[q][1], m.mom[q][2], m.L, K0};
  }
  __device__ __forceinline__ CDF operator()(long long r, int kk) const { return row(r)(kk); }
  __device__ __forceinline__ float2 approx(long long r, int kk) const { return row(r).approx(kk); }
  __device__ __forceinline__ int norm_bits(long long r) const {
    const int q = (int)((r % ((long long)m.np * nv)) / nv);
    return (m.mom[q][0] | m.mom[q][1] | m.mom[q][2]) == 0 ? MS_CAP_B : 0;  // p = 0
  }
};

// phi[u][q][d][i][j] = Phi_acc[u][(d, j)][(q, i)] as complex128, through
// 32 x 32 tiles of (j, i) in shared memory.  Block (32, 8); grid (j tiles,
// i tiles, tb np 7).
__global__ void __launch_bounds__(256) meson_pack_kernel(const CDF* __restrict__ acc, int nv, int np,
                                                         double2* __restrict__ phi) {
  __shared__ double2 tile[32][33];
  const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int z = blockIdx.z;
  const int d = z % MS_NDISP, q = (z / MS_NDISP) % np;
  const long long u = z / (MS_NDISP * np);
  const long long R = (long long)np * nv, M = (long long)MS_NDISP * nv;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int jy = ty; jy < 32; jy += 8) {
    const int j = j0 + jy, i = i0 + tx;
    if (i < nv && j < nv) {
      const CDF v = acc[(u * M + (long long)d * nv + j) * R + (long long)q * nv + i];
      tile[jy][tx] = make_double2(df_to_double(v.re), df_to_double(v.im));
    }
  }
  __syncthreads();
  double2* out = phi + ((u * np + q) * MS_NDISP + d) * (long long)nv * nv;
  for (int iy = ty; iy < 32; iy += 8) {
    const int i = i0 + iy, j = j0 + tx;
    if (i < nv && j < nv) out[(long long)i * nv + j] = tile[tx][iy];
  }
}

// ----------------------------------------------------------- elementals

struct MsElemWs {
  CDF* tab;
  CDF* N;  // displaced fields of the batch [tb][6][nv][V3][3]: nabla_x,y,z, BB_x,y,z
  void *A, *B;
  int *eA, *eB;
  CDF* acc;  // [tb][7 nv][np nv]
};

static MsElemWs carve_melem(Arena& ar, const Scheme& sc, int L, int nv, int np, int tb) {
  const long long V3 = (long long)L * L * L, M = (long long)MS_NDISP * nv, R = (long long)np * nv;
  MsElemWs w;
  w.tab = ar.take<CDF>(L);
  w.N = ar.take<CDF>((size_t)tb * 6 * nv * V3 * 3);
  w.A = ar.take<uint16_t>(tc::plane_img_elems(MS_KC, M, tb, 2 * sc.na));
  w.B = ar.take<uint16_t>(tc::plane_img_elems(MS_KC, R, tb, 2 * sc.nb));
  w.eA = ar.take<int>(tb * M);
  w.eB = ar.take<int>(tb * R);
  w.acc = ar.take<CDF>((size_t)tb * M * R);
  return w;
}

// Timeslices per batch: the one K chunk of one timeslice gives
// ceil(7 N_v / 128) x ceil(N_p N_v / NT) tiles; the batch size with the
// fullest last wave on the SMs (the largest of those within 2 %) among the
// batches whose workspace stays within 16 GiB.
static int meson_elem_batch(const Scheme& sc, int L, int nt, int nv, int np) {
  const long long M = (long long)MS_NDISP * nv, R = (long long)np * nv;
  const int NT = R > 64 ? 80 : 32;
  const long long tiles1 = ((M + 127) / 128) * ((R + NT - 1) / NT);
  Arena one, two;
  carve_melem(one, sc, L, nv, np, 1);
  carve_melem(two, sc, L, nv, np, 2);
  const size_t per = two.used - one.used;
  int best = 1;
  double best_eff = 0.0;
  double eff[4097];
  const int top = nt < 4096 ? nt : 4096;
  for (int tb = 1; tb <= top; ++tb) {
    if (tb > 1 && one.used + (size_t)(tb - 1) * per > (size_t(16) << 30)) break;
    const long long tiles = tiles1 * tb, waves = (tiles + 147) / 148;
    eff[tb] = (double)tiles / (double)(waves * 148);
    if (eff[tb] > best_eff) best_eff = eff[tb];
    best = tb;
  }
  const int last = best;
  for (int tb = last; tb >= 1; --tb)
    if (eff[tb] >= best_eff - 0.02) return tb;
  return 1;
}

size_t meson_elementals_workspace(int L, int nt, int nv, int np) {
  const Scheme sc = elementals_scheme_of(DISTIL_MIXED_FP16X6);
  Arena ar;
  carve_melem(ar, sc, L, nv, np, meson_elem_batch(sc, L, nt, nv, np));
  return ar.used + 256;
}

template <int NT, class Epi>
static int melem_gemm(distil_ctx* ctx, const PlaneImg& A, const PlaneImg& B, const tc::GemmCfg& cfg, int tb,
                      const Epi& epi, cudaStream_t s) {
  return tc::launch_gemm<NT, 16, 8, 8, tc::max_stages<NT, 16, 8, 8>(), false, 3>(ctx, "tc_gemm_meson_elem", A, B,
                                                                               cfg, tb, epi, s);
}

static int melem_batch_run(distil_ctx* ctx, const Scheme& sch, const float2* vt, const float2* Ut, int tb, int L,
                           int nv, const MsMom& mom, double2* phi_t, const MsElemWs& w, cudaStream_t s) {
  constexpr int NA = 4, NB = 4, NPLA = 2 * NA, NPLB = 2 * NB;
  const long long V3 = (long long)L * L * L, Ktot = 3 * V3, M = (long long)MS_NDISP * nv,
                  R = (long long)mom.np * nv;
  const int H = sch.H;
  {
    const long long total = (long long)tb * 3 * nv * V3;
    Launch Ln(ctx, "meson_nabla", s);
    meson_nabla_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(vt, Ut, L, nv, tb, w.N);
  }
  DISTIL_LAUNCH_CHECK();
  {
    const long long total = (long long)tb * nv * V3;
    Launch Lb(ctx, "meson_bb", s);
    meson_bb_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(Ut, L, nv, tb, w.N);
  }
  DISTIL_LAUNCH_CHECK();
  tc::GemmCfg cfg{};
  fill_products(cfg, sch);
  cfg.shift = 2 * H;
  cfg.err = ctx->d_error;
  for (long long K0 = 0; K0 < Ktot; K0 += MS_KC) {
    const int Kc = (int)((Ktot - K0) < MS_KC ? (Ktot - K0) : MS_KC);
    const PlaneImg A = tc::plane_img(w.A, Kc, M, tb, NPLA), B = tc::plane_img(w.B, Kc, R, tb, NPLB);
    DISTIL_TRY((split_rows<false, true, NA>(ctx, "split_meson_disp", DispSrc{vt, w.N, nv, (int)K0, V3},
                                            tb * M, A, H, w.eA, s)));
    DISTIL_TRY((split_rows<false, true, NB>(ctx, "split_meson_phase", PhConjSrc{vt, w.tab, mom, nv, (int)K0, V3},
                                            tb * R, B, H, w.eB, s)));
    cfg.M = (int)M;
    cfg.N = (int)R;
    cfg.K = Kc;
    cfg.a = tc::OpMap{1, tb, 1, 0, 0, (int)M, w.eA};
    cfg.b = tc::OpMap{1, tb, 1, 0, 0, (int)R, w.eB};
    const ColMap cm{1, 0, 0, 0};
    int st;
    if (K0 == 0) {
      EpiStoreCDF epi{{}, w.acc, M * R, 0, 1, R, cm, (int)R};
      st = R > 64 ? melem_gemm<80>(ctx, A, B, cfg, tb, epi, s) : melem_gemm<32>(ctx, A, B, cfg, tb, epi, s);
    } else {
      EpiAddCDF epi{{}, w.acc, M * R, 0, 1, R, cm, (int)R};
      st = R > 64 ? melem_gemm<80>(ctx, A, B, cfg, tb, epi, s) : melem_gemm<32>(ctx, A, B, cfg, tb, epi, s);
    }
    DISTIL_TRY(st);
  }
  {
    Launch Lp(ctx, "meson_pack", s);
    const dim3 grid((unsigned)((nv + 31) / 32), (unsigned)((nv + 31) / 32), (unsigned)(tb * mom.np * MS_NDISP));
    meson_pack_kernel<<<grid, dim3(32, 8), 0, s>>>(w.acc, nv, mom.np, phi_t);
  }
  DISTIL_LAUNCH_CHECK();
  (void)NPLB;
  return DISTIL_OK;
}

int meson_elementals(distil_ctx* ctx, const void* v, const void* U, int L, int nt, int nv, const int32_t* mom,
                     int np, void* phi, void* ws, size_t ws_bytes, cudaStream_t s) {
  const Scheme sch = elementals_scheme_of(DISTIL_MIXED_FP16X6);
  const int tb = meson_elem_batch(sch, L, nt, nv, np);
  Arena ar(ws, ws_bytes);
  MsElemWs w = carve_melem(ar, sch, L, nv, np, tb);
  if (!ar.fits()) {
    set_error("distil_meson_elementals: workspace too small");
    return DISTIL_ENOMEM;
  }
  MsMom m;
  m.np = np;
  m.L = L;
  for (int q = 0; q < np; ++q)
    for (int d = 0; d < 3; ++d) m.mom[q][d] = ((mom[3 * q + d] % L) + L) % L;
  {
    Launch Lz(ctx, "meson_setup", s);
    meson_phase_table_kernel<<<(L + 255) / 256, 256, 0, s>>>(L, w.tab);
  }
  DISTIL_LAUNCH_CHECK();
  const long long V3 = (long long)L * L * L;
  for (int t = 0; t < nt; t += tb) {
    const int n_t = nt - t < tb ? nt - t : tb;
    const float2* vt = reinterpret_cast<const float2*>(v) + (long long)t * nv * V3 * 3;
    const float2* Ut = reinterpret_cast<const float2*>(U) + (long long)t * 3 * V3 * 9;
    double2* pt = reinterpret_cast<double2*>(phi) + (long long)t * np * MS_NDISP * nv * nv;
    DISTIL_TRY(melem_batch_run(ctx, sch, vt, Ut, n_t, L, nv, m, pt, w, s));
  }
  return DISTIL_OK;
}

// ------------------------------------------------------------ correlator

// complex128 -> double-float, optionally transposed and conjugated per
// [nv][nv] block: out[blk][r][c] = in[blk][r][c] or conj(in[blk][c][r]).
__global__ void __launch_bounds__(256) meson_to_cdf_kernel(const double2* __restrict__ in, int nv, int conj_t,
                                                           CDF* __restrict__ out) {
  __shared__ double2 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const long long blk = blockIdx.z;
  const double2* src = in + blk * (long long)nv * nv;
  CDF* dst = out + blk * (long long)nv * nv;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (!conj_t) {
    for (int ry = ty; ry < 32; ry += 8) {
      const int r = r0 + ry, c = c0 + tx;
      if (r < nv && c < nv) {
        const double2 x = src[(long long)r * nv + c];
        dst[(long long)r * nv + c] = cdf_make(df_from_double(x.x), df_from_double(x.y));
      }
    }
    return;
  }
  // read rows c of the tile's columns, write rows r
  for (int ry = ty; ry < 32; ry += 8) {
    const int rr = c0 + ry, cc = r0 + tx;  // element in[rr][cc]
    if (rr < nv && cc < nv) tile[ry][tx] = src[(long long)rr * nv + cc];
  }
  __syncthreads();
  for (int ry = ty; ry < 32; ry += 8) {
    const int r = r0 + ry, c = c0 + tx;  // out[r][c] = conj(in[c][r])
    if (r < nv && c < nv) {
      const double2 x = tile[tx][ry];
      dst[(long long)r * nv + c] = cdf_make(df_from_double(x.x), df_from_double(-x.y));
    }
  }
}

__global__ void meson_prof_kernel(const double* __restrict__ prof, long long n, DF* __restrict__ g) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) g[i] = df_from_double(prof[i]);
}

// displacement of term c of operator type typ
__host__ __device__ __forceinline__ int term_disp(int typ, int c) { return typ == 0 ? 0 : typ == 1 ? 1 + c : 4 + c; }
__host__ __device__ __forceinline__ int term_count(int typ) { return typ == 0 ? 1 : 3; }

// A operand of GEMM 1: row (b, kappa, k) of Phibar_b, K index m = (mu, m'):
//   sum_c [perm_c(kappa) = mu] i^ph_c(kappa) g_k g_m' conj(Phi^(d_c)(0)[m'][k])
// with phiS[d][k][m'] = conj(Phi^d(0)[m'][k]).
struct SrcOpRow {
  const CDF* ph[3];
  int mu[3], phs[3], nc, nv;
  DF gk;
  const DF* g;
  __device__ __forceinline__ CDF operator()(int m) const {
    const int mu_m = m / nv, mp = m - mu_m * nv;
    CDF acc = cdf_zero();
    bool any = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c < nc && mu[c] == mu_m) {
        const CDF z = cdf_iph(ld_cdf(ph[c] + mp), phs[c]);
        acc = any ? cdf_add(acc, z) : z;
        any = true;
      }
    }
    if (!any) return acc;
    return cdf_scale(acc, df_mul(gk, g[mp]));
  }
  __device__ __forceinline__ float2 approx(int m) const {
    const CDF z = (*this)(m);
    return make_float2(z.re.hi, z.im.hi);
  }
};
struct SrcOpSrc {
  const CDF* phiS;  // [np][7][nv][nv]
  const DF* g;      // [nb][nv]
  SpinTab src;
  int nv, nb;
  long long M;      // rows per momentum (3 nb 4 nv)
  __device__ __forceinline__ SrcOpRow row(long long rq) const {
    const long long q = rq / M, r = rq - q * M;
    const CDF* phq = phiS + q * MS_NDISP * (long long)nv * nv;
    const int k = (int)(r % nv);
    const int kap = (int)((r / nv) % 4);
    const int b = (int)(r / (4LL * nv));
    const int typ = b / nb, sg = b - typ * nb;
    SrcOpRow w{};
    w.nc = term_count(typ);
    w.nv = nv;
    w.g = g + (long long)sg * nv;
    w.gk = w.g[k];
    for (int c = 0; c < 3; ++c) {
      const int d = term_disp(typ, c < w.nc ? c : 0);
      w.ph[c] = phq + ((long long)d * nv + k) * nv;
      w.mu[c] = src.perm[d][kap];
      w.phs[c] = src.ph[d][kap];
    }
    return w;
  }
  __device__ __forceinline__ CDF operator()(long long r, int m) const { return row(r)(m); }
  __device__ __forceinline__ float2 approx(long long r, int m) const { return row(r).approx(m); }
};

// B operand of GEMM 1: row L = (lambda, l), K index m = (mu, m'):
//   tau~[m][L] = (g5 tau^dagger g5)[m][L]
//              = i^(ph5(mu) + ph5(p5(lambda))) conj(tau[(p5(lambda), l)][(p5(mu), m')])
// (gamma_5 a real signed involution here)
struct TauTildeRow {
  const float2* trow;  // tau row (p5(lambda), l)
  int p5[4], ph5[4], phl, nv;
  __device__ __forceinline__ CDF operator()(int m) const {
    const int mu = m / nv, mp = m - mu * nv;
    const float2 x = trow[(long long)p5[mu] * nv + mp];
    return cdf_iph(cdf_make(df_make(x.x, 0.f), df_make(-x.y, 0.f)), ph5[mu] + phl);
  }
  __device__ __forceinline__ float2 approx(int m) const {
    const CDF z = (*this)(m);
    return make_float2(z.re.hi, z.im.hi);
  }
};
struct TauTildeSrc {
  const float2* tau;  // [4nv][4nv]
  int p5[4], ph5[4], nv;
  __device__ __forceinline__ TauTildeRow row(long long r) const {
    const int lam = (int)(r / nv), l = (int)(r % nv);
    TauTildeRow w{};
    w.trow = tau + ((long long)p5[lam] * nv + l) * 4 * nv;
    for (int a = 0; a < 4; ++a) {
      w.p5[a] = p5[a];
      w.ph5[a] = ph5[a];
    }
    w.phl = ph5[p5[lam]];
    w.nv = nv;
    return w;
  }
  __device__ __forceinline__ CDF operator()(long long r, int m) const { return row(r)(m); }
  __device__ __forceinline__ float2 approx(long long r, int m) const { return row(r).approx(m); }
};

// rows of a [rows][K] complex64 matrix, exact in double-float (tau for GEMM 2)
struct C64Rows {
  const float2* x;
  long long K;
  __device__ __forceinline__ CDF operator()(long long r, int k) const {
    const float2 v = x[r * K + k];
    return cdf_make(df_make(v.x, 0.f), df_make(v.y, 0.f));
  }
  __device__ __forceinline__ float2 approx(long long r, int k) const { return x[r * K + k]; }
};
// A operand of GEMM 2: row (b, L) = Q_b[.][L] = C1[L][b 4nv + K]
struct QRows {
  const CDF* c1;
  int n4, nops, nb;
  __device__ __forceinline__ int norm_bits(long long r) const { return r / n4 < nb ? MS_CAP_A : 0; }  // type 0
  __device__ __forceinline__ CDF operator()(long long r, int k) const {
    const long long b = r / n4, L = r - b * n4;
    return ld_cdf(c1 + L * ((long long)nops * n4) + b * n4 + k);
  }
  __device__ __forceinline__ float2 approx(long long r, int k) const {
    const CDF z = (*this)(r, k);
    return make_float2(z.re.hi, z.im.hi);
  }
};

// Partial sums of -C_ab over one chunk of i:
//   sum_c sum_alpha i^ph_c(alpha) sum_(i in chunk, j) g_i g_j Phi^(d_c)_ij XT[(b, alpha, i)][(perm_c(alpha), j)]
// for the N_B profiles of type typ at once.  Block (b, typ, chunk), threads
// over j.
constexpr int MS_RED_THREADS = 256;
__global__ void __launch_bounds__(MS_RED_THREADS) meson_reduce_kernel(const CDF* __restrict__ phiC,
                                                                      const CDF* __restrict__ XT,
                                                                      const DF* __restrict__ g, SpinTab snk, int nv,
                                                                      int nb, double2* __restrict__ part) {
  const int b = blockIdx.x, typ = blockIdx.y, chunk = blockIdx.z;
  const int nops = 3 * nb, n4 = 4 * nv;
  const int per = (nv + MS_RED_CHUNKS - 1) / MS_RED_CHUNKS;
  const int i_lo = chunk * per, i_hi = min(nv, i_lo + per);
  const int nc = term_count(typ);
  double tre[MS_MAX_NB], tim[MS_MAX_NB];
#pragma unroll
  for (int s = 0; s < MS_MAX_NB; ++s) tre[s] = tim[s] = 0.0;
  for (int j = threadIdx.x; j < nv; j += MS_RED_THREADS) {
    Dot2 are[MS_MAX_NB], aim[MS_MAX_NB];
    for (int i = i_lo; i < i_hi; ++i) {
      Dot2 wre, wim;
      for (int c = 0; c < nc; ++c) {
        const int d = term_disp(typ, c);
        const CDF f = ld_cdf(phiC + ((long long)d * nv + i) * nv + j);
#pragma unroll
        for (int al = 0; al < 4; ++al) {
          const CDF x = ld_cdf(XT + ((long long)(b * 4 + al) * nv + i) * n4 + (long long)snk.perm[d][al] * nv + j);
          const CDF fx = cdf_iph(f, snk.ph[d][al]);
          wre.add_dd(fx.re, x.re);
          wre.add_dd(df_neg(fx.im), x.im);
          wim.add_dd(fx.re, x.im);
          wim.add_dd(fx.im, x.re);
        }
      }
      const DF wr = wre.get(), wi = wim.get();
#pragma unroll
      for (int s = 0; s < MS_MAX_NB; ++s) {
        if (s < nb) {
          const DF gi = g[(long long)s * nv + i];
          are[s].add_dd(gi, wr);
          aim[s].add_dd(gi, wi);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < MS_MAX_NB; ++s) {
      if (s < nb) {
        const double gj = df_to_double(g[(long long)s * nv + j]);
        tre[s] += gj * df_to_double(are[s].get());
        tim[s] += gj * df_to_double(aim[s].get());
      }
    }
  }
  __shared__ double red[2][MS_MAX_NB][MS_RED_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < MS_MAX_NB; ++s) {
    if (s >= nb) break;
    double x = tre[s], y = tim[s];
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      red[0][s][wid] = x;
      red[1][s][wid] = y;
    }
  }
  __syncthreads();
  if (threadIdx.x < nb) {
    const int s = threadIdx.x;
    double x = 0.0, y = 0.0;
    for (int w = 0; w < MS_RED_THREADS / 32; ++w) {
      x += red[0][s][w];
      y += red[1][s][w];
    }
    part[((long long)chunk * nops + typ * nb + s) * nops + b] = make_double2(x, y);
  }
}

// C[a][b][t] = -sum over chunks (C of one momentum: [nops][nops][nt])
__global__ void meson_final_kernel(const double2* __restrict__ part, int nops, int nt, int t, double2* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nops * nops) return;
  double x = 0.0, y = 0.0;
  for (int c = 0; c < MS_RED_CHUNKS; ++c) {
    const double2 p = part[(long long)c * nops * nops + e];
    x += p.x;
    y += p.y;
  }
  C[(long long)e * nt + t] = make_double2(-x, -y);
}

struct MsCorrWs {
  DF* g;
  CDF *phiS, *phiC;
  void *A1, *B1, *A2, *B2;
  int *eA1, *eB1, *eA2, *eB2;
  CDF *C1, *XT;
  double2* part;
};

static MsCorrWs carve_mcorr(Arena& ar, const Scheme& sc, int nv, int np, int nb) {
  const long long n4 = 4LL * nv, nops = 3LL * nb, M = nops * n4;
  MsCorrWs w;
  w.g = ar.take<DF>((size_t)nb * nv);
  w.phiS = ar.take<CDF>((size_t)np * MS_NDISP * nv * nv);
  w.phiC = ar.take<CDF>((size_t)np * MS_NDISP * nv * nv);
  w.A1 = ar.take<uint16_t>(tc::plane_img_elems(n4, M, np, 2 * sc.na));
  w.B1 = ar.take<uint16_t>(tc::plane_img_elems(n4, n4, 1, 2 * sc.nb));
  w.A2 = ar.take<uint16_t>(tc::plane_img_elems(n4, M, 1, 2 * sc.na));
  w.B2 = ar.take<uint16_t>(tc::plane_img_elems(n4, n4, 1, 2 * sc.nb));
  w.eA1 = ar.take<int>(np * M);
  w.eB1 = ar.take<int>(n4);
  w.eA2 = ar.take<int>(M);
  w.eB2 = ar.take<int>(n4);
  w.C1 = ar.take<CDF>((size_t)M * n4);
  w.XT = ar.take<CDF>((size_t)M * n4);
  w.part = ar.take<double2>((size_t)MS_RED_CHUNKS * nops * nops);
  return w;
}

size_t meson_correlate_workspace(int nv, int np, int nb) {
  Arena ar;
  carve_mcorr(ar, scheme_of(DISTIL_MIXED_FP16X6), nv, np, nb);
  return ar.used + 256;
}

// 80-wide tiles on the persistent kernel with one accumulator set (the MMAs
// of a tile wait for the previous tile's epilogue while the copies of the
// next run; K = 4 N_v is short, so the epilogue of one tile per CTA would
// otherwise sit between the copies); 32-wide one-tile launches for N <= 64.
template <int NT>
static int mcorr_gemm(distil_ctx* ctx, const char* name, const PlaneImg& A, const PlaneImg& B,
                      const tc::GemmCfg& cfg, const EpiStoreCDF& epi, cudaStream_t s) {
  if constexpr (NT == 80)
    return tc::launch_gemm_persistent<80, 16, 6, 8, tc::max_stages<80, 16, 6, 8>(), false, 3, 1>(ctx, name, A, B,
                                                                                               cfg, 1, epi, s);
  else
    return tc::launch_gemm<NT, 16, 6, 8, tc::max_stages<NT, 16, 6, 8>(), false, 3>(ctx, name, A, B, cfg, 1, epi, s);
}

int meson_correlate(distil_ctx* ctx, const void* phi_snk, const void* phi_src, const void* tau, int nt, int nv,
                    int np, const double* prof, int nb, void* C, void* ws, size_t ws_bytes, cudaStream_t s) {
  constexpr int NA = 3, NB = 4, NPLA = 2 * NA, NPLB = 2 * NB;
  SpinTabs sp;
  if (!spin_tables(sp)) {
    set_error("distil_meson_correlate: gamma matrices are not signed permutations");
    return DISTIL_EINVAL;
  }
  const Scheme sch = scheme_of(DISTIL_MIXED_FP16X6);
  Arena ar(ws, ws_bytes);
  MsCorrWs w = carve_mcorr(ar, sch, nv, np, nb);
  if (!ar.fits()) {
    set_error("distil_meson_correlate: workspace too small");
    return DISTIL_ENOMEM;
  }
  const int n4 = 4 * nv, nops = 3 * nb;
  const long long M = (long long)nops * n4, blk = (long long)nv * nv;
  // fixed-point leading slice as for the public split GEMM (K = 4 N_v)
  const int H = n4 <= 1024 ? sch.H : n4 <= 4096 ? 9 : n4 <= 16384 ? 8 : 7;
  const dim3 tgrid((unsigned)((nv + 31) / 32), (unsigned)((nv + 31) / 32), (unsigned)(np * MS_NDISP));
  {
    Launch Lp(ctx, "meson_corr_setup", s);
    meson_prof_kernel<<<(unsigned)(((long long)nb * nv + 255) / 256), 256, 0, s>>>(prof, (long long)nb * nv, w.g);
    meson_to_cdf_kernel<<<tgrid, dim3(32, 8), 0, s>>>((const double2*)phi_src, nv, 1, w.phiS);
  }
  DISTIL_LAUNCH_CHECK();
  tc::GemmCfg cfg{};
  fill_products(cfg, sch);
  cfg.shift = 2 * H;
  cfg.err = ctx->d_error;
  cfg.K = n4;
  // source operands of GEMM 1, image coordinate q for momentum q
  const PlaneImg A1 = tc::plane_img(w.A1, n4, M, np, NPLA);
  DISTIL_TRY((split_rows<false, true, NA>(ctx, "split_meson_srcop", SrcOpSrc{w.phiS, w.g, sp.src, nv, nb, M},
                                          (long long)np * M, A1, H, w.eA1, s)));
  const PlaneImg B1 = tc::plane_img(w.B1, n4, n4, 1, NPLB), A2 = tc::plane_img(w.A2, n4, M, 1, NPLA),
                 B2 = tc::plane_img(w.B2, n4, n4, 1, NPLB);
  TauTildeSrc tts{};
  for (int a = 0; a < 4; ++a) {
    tts.p5[a] = sp.g5perm[a];
    tts.ph5[a] = sp.g5ph[a];
  }
  tts.nv = nv;
  for (int t = 0; t < nt; ++t) {
    const float2* tau_t = reinterpret_cast<const float2*>(tau) + (long long)t * n4 * n4;
    tts.tau = tau_t;
    DISTIL_TRY((split_rows<false, true, NB>(ctx, "split_meson_tautilde", tts, n4, B1, H, w.eB1, s)));
    DISTIL_TRY((split_rows<false, true, NB>(ctx, "split_meson_tau", C64Rows{tau_t, n4}, n4, B2, H, w.eB2, s,
                                            nullptr, MS_CAP_B)));
    {
      Launch Lc(ctx, "meson_corr_setup", s);
      meson_to_cdf_kernel<<<tgrid, dim3(32, 8), 0, s>>>(
          reinterpret_cast<const double2*>(phi_snk) + (long long)t * np * MS_NDISP * blk, nv, 0, w.phiC);
    }
    DISTIL_LAUNCH_CHECK();
    for (int q = 0; q < np; ++q) {
      // GEMM 1: D[(b, K)][L] = (Phibar_b tau~)[K][L], stored C1[L][(b, K)]
      cfg.M = (int)M;
      cfg.N = n4;
      cfg.a = tc::OpMap{1, 1, 1, q, 0, (int)M, w.eA1};
      cfg.b = tc::OpMap{1, 1, 1, 0, 0, n4, w.eB1};
      {
        EpiStoreCDF epi{{}, w.C1, 0, 0, 1, 1, ColMap{M, 0, 0, 0}, n4};
        DISTIL_TRY(n4 > 64 ? mcorr_gemm<80>(ctx, "tc_gemm_meson_q", A1, B1, cfg, epi, s)
                           : mcorr_gemm<32>(ctx, "tc_gemm_meson_q", A1, B1, cfg, epi, s));
      }
      // GEMM 2: D[(b, L)][I] = (tau Q_b)[I][L] = X_b[I][L], stored XT[(b, L)][I]
      DISTIL_TRY((split_rows<false, true, NA>(ctx, "split_meson_q", QRows{w.C1, n4, nops, nb}, M, A2, H, w.eA2, s)));
      cfg.a = tc::OpMap{1, 1, 1, 0, 0, (int)M, w.eA2};
      cfg.b = tc::OpMap{1, 1, 1, 0, 0, n4, w.eB2};
      {
        EpiStoreCDF epi{{}, w.XT, 0, 0, 1, n4, ColMap{1, 0, 0, 0}, n4};
        DISTIL_TRY(n4 > 64 ? mcorr_gemm<80>(ctx, "tc_gemm_meson_x", A2, B2, cfg, epi, s)
                           : mcorr_gemm<32>(ctx, "tc_gemm_meson_x", A2, B2, cfg, epi, s));
      }
      {
        Launch Lr(ctx, "meson_reduce", s);
        meson_reduce_kernel<<<dim3((unsigned)nops, 3, MS_RED_CHUNKS), MS_RED_THREADS, 0, s>>>(
            w.phiC + (long long)q * MS_NDISP * blk, w.XT, w.g, sp.snk, nv, nb, w.part);
        meson_final_kernel<<<(nops * nops + 127) / 128, 128, 0, s>>>(
            w.part, nops, nt, t, reinterpret_cast<double2*>(C) + (long long)q * nops * nops * nt);
      }
      DISTIL_LAUNCH_CHECK();
    }
  }
  return DISTIL_OK;
}

// --------------------------------------------------------------- pruning

// One-sided (Hestenes) Jacobi SVD of A = C(t_p) (nops <= 32 columns, lane =
// row): column pairs are rotated until orthogonal, A V = W; the singular
// values are the column norms of W and the left singular vectors its
// normalised columns.  The pairs of a sweep run in the round-robin
// (circle) order, the n/2 disjoint pairs of a round on n/2 warps at once.
// Output: the n columns of the largest singular values, each scaled so that
// its largest-modulus component (the first of equal ones) is real and
// positive, and all singular values, descending.
constexpr int MS_SVD_WARPS = 16;
__global__ void __launch_bounds__(32 * MS_SVD_WARPS) meson_svd_kernel(const double2* __restrict__ C, int nops, int nt,
                                                                      int tp, int nkeep, double2* __restrict__ Un,
                                                                      double* __restrict__ sv) {
  __shared__ double2 A[32][33];
  __shared__ double nrm[32], offw[MS_SVD_WARPS];
  __shared__ int order[32];
  __shared__ int done;
  const int q = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double2* Cq = C + (long long)q * nops * nops * nt;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    A[r][c] = (r < nops && c < nops) ? Cq[((long long)r * nops + c) * nt + tp] : make_double2(0.0, 0.0);
  }
  const int n = (nops + 1) & ~1;  // even number of columns for the circle order
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  for (int sweep = 0; sweep < 40 && !done; ++sweep) {
    double off = 0.0;  // largest |a_p^H a_r| / (|a_p| |a_r|) this warp met
    for (int round = 0; round < n - 1; ++round) {
      if (w < n / 2) {
        int p, r;
        if (w == 0) {
          p = round;
          r = n - 1;
        } else {
          p = (round + w) % (n - 1);
          r = (round - w + n - 1) % (n - 1);
        }
        if (p > r) {
          const int x = p;
          p = r;
          r = x;
        }
        if (r < nops) {
          const double2 ap = A[lane][p], ar = A[lane][r];
          double al = ap.x * ap.x + ap.y * ap.y, be = ar.x * ar.x + ar.y * ar.y;
          double gr = ap.x * ar.x + ap.y * ar.y, gi = ap.x * ar.y - ap.y * ar.x;  // conj(ap) ar
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            gr += __shfl_xor_sync(0xffffffffu, gr, o);
            gi += __shfl_xor_sync(0xffffffffu, gi, o);
          }
          const double ga = sqrt(gr * gr + gi * gi);
          const double nab = sqrt(al * be);
          if (nab > 0.0) off = fmax(off, ga / nab);
          if (ga > 1e-15 * nab) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
            const double er = gr / ga, ei = gi / ga;  // e^{i phi}
            // a_p' = c a_p - s e^{-i phi} a_r,  a_r' = s e^{i phi} a_p + c a_r
            A[lane][p] = make_double2(c * ap.x - s * (er * ar.x + ei * ar.y), c * ap.y - s * (er * ar.y - ei * ar.x));
            A[lane][r] = make_double2(s * (er * ap.x - ei * ap.y) + c * ar.x, s * (er * ap.y + ei * ap.x) + c * ar.y);
          }
        }
      }
      __syncthreads();
    }
    if (lane == 0) offw[w] = off;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int k = 0; k < MS_SVD_WARPS; ++k) m = fmax(m, offw[k]);
      done = m < 1e-13;  // columns orthogonal to well below the FP64 rounding of the data
    }
    __syncthreads();
  }
  if (w != 0) return;
  if (lane < nops) {
    double s2 = 0.0;
    for (int r = 0; r < nops; ++r) s2 += A[r][lane].x * A[r][lane].x + A[r][lane].y * A[r][lane].y;
    nrm[lane] = sqrt(s2);
  }
  __syncwarp();
  if (lane == 0) {
    for (int c = 0; c < nops; ++c) order[c] = c;
    for (int a = 0; a < nops; ++a)  // selection sort, descending, stable
      for (int b = a + 1; b < nops; ++b)
        if (nrm[order[b]] > nrm[order[a]]) {
          const int x = order[a];
          order[a] = order[b];
          order[b] = x;
        }
  }
  __syncwarp();
  if (lane < nops && sv) sv[(long long)q * nops + lane] = nrm[order[lane]];
  for (int m = 0; m < nkeep; ++m) {
    const int c = order[m];
    const double nm = nrm[c];
    double2 u = lane < nops && nm > 0.0 ? make_double2(A[lane][c].x / nm, A[lane][c].y / nm) : make_double2(0.0, 0.0);
    // phase: the largest-modulus component (first of equal ones) real positive
    double best = lane < nops ? u.x * u.x + u.y * u.y : -1.0;
    int arg = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
    }
    const double kx = __shfl_sync(0xffffffffu, u.x, arg), ky = __shfl_sync(0xffffffffu, u.y, arg);
    const double km = sqrt(kx * kx + ky * ky);
    if (km > 0.0) {
      const double cr = kx / km, ci = -ky / km;  // conj(u_k) / |u_k|
      u = make_double2(u.x * cr - u.y * ci, u.x * ci + u.y * cr);
    }
    if (lane < nops) Un[((long long)q * nops + lane) * nkeep + m] = u;
  }
}

// Ct[q][m][n][t] = sum_ab conj(U[a][m]) C[q][a][b][t] U[b][n]; block (q, t)
__global__ void __launch_bounds__(256) meson_project_kernel(const double2* __restrict__ C,
                                                            const double2* __restrict__ Un, int nops, int nt,
                                                            int nkeep, double2* __restrict__ Ct) {
  __shared__ double2 Cs[32][33], Us[32][16], Y[32][16];
  const int q = blockIdx.x, t = blockIdx.y;
  const double2* Cq = C + (long long)q * nops * nops * nt;
  for (int e = threadIdx.x; e < nops * nops; e += blockDim.x) Cs[e / nops][e % nops] = Cq[(long long)e * nt + t];
  for (int e = threadIdx.x; e < nops * nkeep; e += blockDim.x)
    Us[e / nkeep][e % nkeep] = Un[(long long)q * nops * nkeep + e];
  __syncthreads();
  for (int e = threadIdx.x; e < nops * nkeep; e += blockDim.x) {  // Y = C U
    const int a = e / nkeep, n = e % nkeep;
    double x = 0.0, y = 0.0;
    for (int b = 0; b < nops; ++b) {
      const double2 c = Cs[a][b], u = Us[b][n];
      x += c.x * u.x - c.y * u.y;
      y += c.x * u.y + c.y * u.x;
    }
    Y[a][n] = make_double2(x, y);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nkeep * nkeep; e += blockDim.x) {  // U^dagger Y
    const int m = e / nkeep, n = e % nkeep;
    double x = 0.0, y = 0.0;
    for (int a = 0; a < nops; ++a) {
      const double2 u = Us[a][m], z = Y[a][n];
      x += u.x * z.x + u.y * z.y;
      y += u.x * z.y - u.y * z.x;
    }
    Ct[(((long long)q * nkeep + m) * nkeep + n) * nt + t] = make_double2(x, y);
  }
}

int meson_prune(distil_ctx* ctx, const void* C, int np, int nops, int nt, int tp, int nkeep, void* Ct, void* Un,
                double* sv, cudaStream_t s) {
  {
    Launch L(ctx, "meson_prune", s);
    meson_svd_kernel<<<np, 32 * MS_SVD_WARPS, 0, s>>>((const double2*)C, nops, nt, tp, nkeep, (double2*)Un, sv);
    meson_project_kernel<<<dim3(np, nt), 256, 0, s>>>((const double2*)C, (const double2*)Un, nops, nt, nkeep,
                                                      (double2*)Ct);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}


}  // namespace distil
