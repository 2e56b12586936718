// Mixed-precision nucleon elementals on tcgen05 tensor cores.
//
//   Phi[t][q]_ijk = sum_(x,a) E_(i,q)(x,a) W_(j,k)(x,a),
//   E_(i,q)(x,a) = exp(-i p_q.x) v_i^a(x),   W_(j,k) = v_j x v_k (colour cross product)
//
// per timeslice as one complex GEMM with M = pairs j<k (ordered by j, then
// k), N = (i, q) rows and K = (site, colour) (FP16X6: 4 x 4 fixed-point
// pieces, eight products, elementals_scheme_of).  K is cut into chunks of
// EL_KC values: per chunk the operands are formed from the eigenvectors in
// double-float arithmetic (the cross products exactly, by TwoProduct) and
// split into 16-bit pieces with per-(row, chunk) exponents; the tensor
// cores accumulate the chunk in TMEM (the leading fixed-point slice
// exactly), and the epilogue adds the chunk into a double-float accumulator
// Phi_acc[(i,q)][pair] (pairs contiguous, so the 32 rows of an epilogue
// warp read and write 512 contiguous bytes).  Tiles whose every i is >= every j are skipped.  A
// final pass packs i<j<k into Phi[t][q][rank] as complex128.
#include <math.h>

#include "df.cuh"
#include "elementals.cuh"
#include "mixed.cuh"
#include "mixed_common.cuh"

namespace distil {

using tc::PlaneImg;

// K values per accumulation chunk: whole sites (a multiple of 3) and whole
// 16-value K blocks of the plane images, so a chunk holds sites
// [K0/3, (K0 + EL_KC)/3).
constexpr int EL_KC = 4032;
static_assert(EL_KC % 3 == 0 && EL_KC % 16 == 0, "chunks of whole sites and K blocks");

// pairs in j-major order: q -> (j, k), first index j, then k = j+1..n-1
__host__ __device__ __forceinline__ long long jmajor_first(long long j, long long n) { return j * (2 * n - j - 1) / 2; }
__global__ void pair_table_kernel(int n, int2* pairs) {
  const long long P2 = comb2(n);
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= P2) return;
  const float b = 2.f * n - 1.f;
  long long j = (long long)floorf((b - sqrtf(fmaxf(b * b - 8.f * (float)q, 0.f))) * 0.5f);
  if (j < 0) j = 0;
  while (j > 0 && jmajor_first(j, n) > q) --j;
  while (jmajor_first(j + 1, n) <= q) ++j;
  pairs[q] = make_int2((int)j, (int)(q - jmajor_first(j, n) + j + 1));
}

// exp(-2 pi i m / L) as double-floats
__global__ void phase_table_kernel(int L, CDF* tab) {
  const int m = threadIdx.x + blockIdx.x * blockDim.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)L, &s, &c);
  tab[m] = cdf_make(df_from_double(c), df_from_double(-s));
}

struct MomArgs {
  int np, L;
  int mom[EL_MAX_MOM][3];
};

// w^a(x) = v_j^b(x) v_k^c(x) - v_j^c(x) v_k^b(x) for K = 3 x + a, exactly as
// a double-float, from the two eigenvector rows of a pair
struct WRow {
  const float2 *vj, *vk;
  int K0;
  __device__ __forceinline__ CDF operator()(int kk) const {
    const int K = K0 + kk;
    const int x = K / 3, a = K - 3 * x;
    const int b = a == 2 ? 0 : a + 1, c = a == 0 ? 2 : a - 1;
    const float2 jb = vj[3 * x + b], jc = vj[3 * x + c], kb = vk[3 * x + b], kc = vk[3 * x + c];
    const DF re = dot4(jb.x, kc.x, -jb.y, kc.y, -jc.x, kb.x, jc.y, kb.y);
    const DF im = dot4(jb.x, kc.y, jb.y, kc.x, -jc.x, kb.y, -jc.y, kb.x);
    return cdf_make(re, im);
  }
  __device__ __forceinline__ float2 approx(int kk) const {
    const CDF z = (*this)(kk);
    return make_float2(z.re.hi, z.im.hi);
  }
};
struct WSrc {  // rows u P2 + q (timeslice u of the batch, pair q), K = (x, a) from K0 (3 V3 < 2^31)
  const float2* v;  // v[u] = [n][V3][3], stride vs
  const int2* pairs;
  long long V3, P2, vs;
  int K0;
  __device__ __forceinline__ WRow row(long long r) const {
    const long long u = r / P2, q = r - u * P2;
    const int2 jk = pairs[q];
    const float2* vu = v + u * vs;
    return WRow{vu + (long long)jk.x * V3 * 3, vu + (long long)jk.y * V3 * 3, K0};
  }
  __device__ __forceinline__ CDF operator()(long long r, int kk) const { return row(r)(kk); }
  __device__ __forceinline__ float2 approx(long long r, int kk) const { return row(r).approx(kk); }
};

// exp(-i p_q . x) v_i^a(x) for K = 3 x + a, from one eigenvector row
struct ERow {
  const float2* vi;
  const CDF* tab;
  int m0, m1, m2, L, K0;
  __device__ __forceinline__ CDF operator()(int kk) const {
    const int K = K0 + kk;
    const int x = K / 3, a = K - 3 * x;
    const int xy = x / L, xs = x - xy * L, zs = xy / L, ys = xy - zs * L;
    const int ph = (m0 * xs + m1 * ys + m2 * zs) % L;
    const CDF e = tab[ph];
    const float2 u = vi[3 * x + a];
    // (e.re + i e.im)(u.x + i u.y)
    return cdf_make(df_sub(df_mul_f(e.re, u.x), df_mul_f(e.im, u.y)), df_add(df_mul_f(e.re, u.y), df_mul_f(e.im, u.x)));
  }
  __device__ __forceinline__ float2 approx(int kk) const {
    const CDF z = (*this)(kk);
    return make_float2(z.re.hi, z.im.hi);
  }
};
struct ESrc {  // rows u R + i*np + q (timeslice u of the batch), K = (x, a) from K0 (3 V3 < 2^31)
  const float2* v;  // v[u], stride vs
  const CDF* tab;
  MomArgs m;
  long long V3, R, vs;
  int K0;
  __device__ __forceinline__ ERow row(long long rr) const {
    const long long ts = rr / R;
    const int r = (int)(rr - ts * R);
    const int i = r / m.np, q = r - i * m.np;
    return ERow{v + ts * vs + (long long)i * V3 * 3, tab, m.mom[q][0], m.mom[q][1], m.mom[q][2], m.L, K0};
  }
  __device__ __forceinline__ CDF operator()(long long r, int kk) const { return row(r)(kk); }
  __device__ __forceinline__ float2 approx(long long r, int kk) const { return row(r).approx(kk); }
};

// Phi_acc[r][q] (+)= D for the pair rows q and (i, q') columns r; the first
// chunk stores.  Tiles with min i >= max j hold no kept output.
struct EpiPhiAcc : tc::EpiStateless {
  CDF* acc;              // [batch][R][P2]
  const int2* pairs;
  long long P2;
  int N, np, first, nt;  // nt: N tile width of the launch
  __device__ __forceinline__ bool skip_tile(int m_tile, int n_tile, int) const {
    long long qlast = (long long)m_tile * 128 + 127;
    if (qlast >= P2) qlast = P2 - 1;
    const int jmax = pairs[qlast].x;       // j never decreases along the pair order
    const int imin = (n_tile * nt) / np;   // rows are i * np + q
    return imin >= jmax;
  }
  __device__ __forceinline__ void operator()(State&, int batch, int row, int col0, const float* re0,
                                             const float* re1, const float* im0, const float* im1) const {
    CDF* dst = acc + ((long long)batch * N + col0) * P2 + row;
    // all 16 loads in flight before the first store (the stores could
    // otherwise alias the later loads and serialise the round trips)
    CDF old[16];
    if (!first) {
#pragma unroll
      for (int e = 0; e < 16; ++e) old[e] = col0 + e < N ? ld_cdf(dst + e * P2) : cdf_zero();
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if (col0 + e >= N) break;
      CDF v = cdf_make(two_sum(re0[e], re1[e]), two_sum(im0[e], im1[e]));
      if (!first) v = cdf_add(v, old[e]);
      dst[e * P2] = v;
    }
  }
};

// Phi[q][rank(i,j,k)] = Phi_acc[i*np + q][pair(j,k)]  (complex128), i < j,
// through 32 x 32 tiles of (i, pair) in shared memory: the accumulator is
// read along the pairs and Phi written along i (consecutive ranks).
// Block (32, 8) threads; grid (pair tiles, i tiles, np).
__global__ void __launch_bounds__(256) pack_phi_kernel(const CDF* __restrict__ acc, const int2* __restrict__ pairs,
                                                       int n, int np, double2* __restrict__ phi) {
  __shared__ double2 tile[32][33];
  const long long P2 = comb2(n), T3 = comb3(n);
  const long long p0 = (long long)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32, q = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int iy = ty; iy < 32; iy += 8) {
    const int i = i0 + iy;
    const long long pr = p0 + tx;
    if (i < n && pr < P2) {
      const CDF v = acc[((long long)i * np + q) * P2 + pr];
      tile[iy][tx] = make_double2(df_to_double(v.re), df_to_double(v.im));
    }
  }
  __syncthreads();
  double2* out = phi + (long long)q * T3;
  for (int py = ty; py < 32; py += 8) {
    const long long pr = p0 + py;
    if (pr >= P2) break;
    const int2 jk = pairs[pr];
    const int i = i0 + tx;
    if (i < jk.x) out[triple_rank(i, jk.x, jk.y)] = tile[tx][py];
  }
}

struct ElemWs {
  int2* pairs;
  CDF* tab;
  void *W, *E;  // plane images of one K chunk (cross products, phases)
  int *eW, *eE;
  CDF* acc;
};

static ElemWs carve_elem(Arena& ar, const Scheme& sc, int L, int nv, int np, int tb) {
  const long long P2 = comb2(nv), R = (long long)nv * np;
  ElemWs w;
  w.pairs = ar.take<int2>(P2 > 0 ? P2 : 1);
  w.tab = ar.take<CDF>(L);
  w.W = ar.take<uint16_t>(tc::plane_img_elems(EL_KC, P2, tb, 2 * sc.na));
  w.E = ar.take<uint16_t>(tc::plane_img_elems(EL_KC, R, tb, 2 * sc.nb));
  w.eW = ar.take<int>(tb * (P2 > 0 ? P2 : 1));
  w.eE = ar.take<int>(tb * R);
  w.acc = ar.take<CDF>(tb * P2 * R);
  return w;
}

// Timeslices per GEMM launch: one timeslice's K chunk gives (P2 / 128) x
// (R / NT) tiles, of which the triangle skip keeps about 40 %; below about
// eight waves of tiles on the SMs the last wave leaves many SMs idle, so
// small N_v batch several timeslices (each its own accumulator) into every
// launch, as many as keep the batch's operands and accumulators within 4 GiB.
static int elem_batch(const Scheme& sc, int L, int nt, int nv, int np) {
  const long long P2 = comb2(nv), R = (long long)nv * np;
  const long long tiles = ((P2 + 127) / 128) * ((R + 79) / 80);
  const long long kept = tiles * 2 / 5 + 1;
  long long tb = (8LL * 148 + kept - 1) / kept;
  if (tb > nt) tb = nt;
  Arena one, two;
  carve_elem(one, sc, L, nv, np, 1);
  carve_elem(two, sc, L, nv, np, 2);
  const size_t per = two.used - one.used;
  while (tb > 1 && one.used + (size_t)(tb - 1) * per > (size_t(4) << 30)) --tb;
  return tb < 1 ? 1 : (int)tb;
}

size_t elementals_mixed_workspace(int L, int nt, int nv, int np, int mode) {
  const Scheme sc = elementals_scheme_of(mode);
  Arena ar;
  carve_elem(ar, sc, L, nv, np, elem_batch(sc, L, nt, nv, np));
  return ar.used + 256;
}

// The elementals of tb consecutive timeslices (v of the first at vt, Phi of
// the first at phi_t), every GEMM launch covering all tb of them.
template <bool BF16, bool FIXED, int NA, int NB>
static int elem_t(distil_ctx* ctx, const Scheme& sch, int H, const float2* vt, int tb, int L, int nv,
                  const MomArgs& mom, double2* phi_t, const ElemWs& w, cudaStream_t s) {
  constexpr int NPLA = 2 * NA, NPLB = 2 * NB;
  const long long V3 = (long long)L * L * L, Ktot = 3 * V3, P2 = comb2(nv), R = (long long)nv * mom.np;
  const long long vs = (long long)nv * V3 * 3;
  tc::GemmCfg cfg{};
  fill_products(cfg, sch);
  cfg.shift = 2 * H;
  cfg.err = ctx->d_error;
  for (long long K0 = 0; K0 < Ktot; K0 += EL_KC) {
    const int Kc = (int)((Ktot - K0) < EL_KC ? (Ktot - K0) : EL_KC);
    const tc::PlaneImg A = tc::plane_img(w.W, Kc, P2, tb, NPLA), B = tc::plane_img(w.E, Kc, R, tb, NPLB);
    DISTIL_TRY((split_rows<BF16, FIXED, NA>(ctx, "split_pairs", WSrc{vt, w.pairs, V3, P2, vs, (int)K0}, tb * P2, A, H,
                                            w.eW, s)));
    DISTIL_TRY((split_rows<BF16, FIXED, NB>(ctx, "split_phase", ESrc{vt, w.tab, mom, V3, R, vs, (int)K0}, tb * R, B, H,
                                            w.eE, s)));
    cfg.M = (int)P2; cfg.N = (int)R; cfg.K = Kc;
    cfg.a = tc::OpMap{1, tb, 1, 0, 0, (int)P2, w.eW};
    cfg.b = tc::OpMap{1, tb, 1, 0, 0, (int)R, w.eE};
    EpiPhiAcc epi{{}, w.acc, w.pairs, P2, (int)R, mom.np, K0 == 0 ? 1 : 0, 128};
    // K = 4032 per chunk: a deep ring of 16-wide K steps keeps enough of the
    // operand stream (the A pieces come from HBM) in flight.  The 6-product
    // schemes accumulate in three pairs (exact cross terms), which leaves
    // TMEM room for 80-wide N tiles.
    constexpr int NACC = NPLA >= 6 ? 3 : 2;
    constexpr int NTW = NACC == 3 ? 80 : 128;
    constexpr int ST = tc::max_stages<NTW, 16, NPLA, NPLB>();
    int st;
    if (R > 64) {
      epi.nt = NTW;
      // one tile per CTA: the hardware hands out the tiles that survive the
      // triangle skip as SMs free up (a persistent kernel's static tile
      // assignment balanced them worse: 531 against 481 ms per L = 48 step)
      st = tc::launch_gemm<NTW, 16, NPLA, NPLB, ST, BF16, NACC>(ctx, "tc_gemm_elementals", A, B, cfg, tb, epi, s);
    } else if (R > 32) {
      epi.nt = 64;
      st = tc::launch_gemm<64, 16, NPLA, NPLB, tc::max_stages<64, 16, NPLA, NPLB>(), BF16, NACC>(
          ctx, "tc_gemm_elementals", A, B, cfg, tb, epi, s);
    } else {
      epi.nt = 32;
      st = tc::launch_gemm<32, 16, NPLA, NPLB, tc::max_stages<32, 16, NPLA, NPLB>(), BF16, NACC>(
          ctx, "tc_gemm_elementals", A, B, cfg, tb, epi, s);
    }
    DISTIL_TRY(st);
  }
  {
    Launch Lz(ctx, "pack_phi", s);
    const dim3 grid((unsigned)((comb2(nv) + 31) / 32), (unsigned)((nv + 31) / 32), (unsigned)mom.np);
    for (int u = 0; u < tb; ++u)
      pack_phi_kernel<<<grid, dim3(32, 8), 0, s>>>(w.acc + (long long)u * R * P2, w.pairs, nv, mom.np,
                                                  phi_t + (long long)u * mom.np * comb3(nv));
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

int elementals_mixed(distil_ctx* ctx, const Cx<float>* v, int L, int nt, int nv, const int32_t* mom, int np,
                     int mode, void* phi, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (comb3(nv) == 0) return DISTIL_OK;
  const Scheme sch = elementals_scheme_of(mode);
  Arena ar(ws, ws_bytes);
  ElemWs w = carve_elem(ar, sch, L, nv, np, elem_batch(sch, L, nt, nv, np));
  if (!ar.fits()) {
    set_error("distil_elementals: workspace too small");
    return DISTIL_ENOMEM;
  }
  MomArgs m;
  m.np = np;
  m.L = L;
  for (int q = 0; q < np; ++q)
    for (int d = 0; d < 3; ++d) m.mom[q][d] = ((mom[3 * q + d] % L) + L) % L;
  {
    Launch Lz(ctx, "elementals_setup", s);
    pair_table_kernel<<<(unsigned)((comb2(nv) + 255) / 256), 256, 0, s>>>(nv, w.pairs);
    phase_table_kernel<<<(L + 255) / 256, 256, 0, s>>>(L, w.tab);
  }
  DISTIL_LAUNCH_CHECK();
  const long long V3 = (long long)L * L * L, T3 = comb3(nv);
  const int H = sch.H;
  const int tb = elem_batch(sch, L, nt, nv, np);
  for (int t = 0; t < nt; t += tb) {
    const int n_t = nt - t < tb ? nt - t : tb;
    const float2* vt = reinterpret_cast<const float2*>(v) + (long long)t * nv * V3 * 3;
    double2* pt = reinterpret_cast<double2*>(phi) + (long long)t * np * T3;
    int st;
    if (mode == DISTIL_MIXED_FP16X6)
      st = elem_t<false, true, 4, 4>(ctx, sch, H, vt, n_t, L, nv, m, pt, w, s);
    else if (mode == DISTIL_MIXED_BF16X6)
      st = elem_t<true, true, 3, 4>(ctx, sch, H, vt, n_t, L, nv, m, pt, w, s);
    else if (mode == DISTIL_MIXED_BF16X3)
      st = elem_t<true, true, 2, 2>(ctx, sch, H, vt, n_t, L, nv, m, pt, w, s);
    else
      st = elem_t<false, false, 2, 2>(ctx, sch, H, vt, n_t, L, nv, m, pt, w, s);
    if (st != DISTIL_OK) return st;
  }
  return DISTIL_OK;
}

}  // namespace distil
