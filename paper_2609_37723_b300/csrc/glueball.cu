// A1^{-+} glueball operators from the chromo-magnetic field and adjoint
// covariant derivatives (paper Sec. 2.2, "Improved glueball operators"), in
// FP64 on CUDA cores:
//
//  F_{mu nu}(x) = (Q - Q^dag) / (8 i) - (its trace) / 3, Q the four
//                 plaquettes of the (mu, nu) plane that start and end at x
//                 (the clover), B_i = eps_ijk F_jk = 2 F_jk ((i, j, k) cyclic);
//  (D_j X)(x)   = 1/2 [U_j(x) X(x+j) U_j(x)^dag - U_j(x-j)^dag X(x-j) U_j(x-j)];
//  O_1 = sum_x Tr(eps_ijk B_i D_j B_k)          O_2 = sum_x Tr(eps_ijk eps_ilm B_j B_k D_l B_m)
//  O_3 = sum_x Tr(eps_ijk B_i D_j^3 B_k)        O_4 = sum_x Tr(eps_ijk B_i D_j^2 D_k B_j)
//  O_5 = sum_x Tr(eps_ijk B_i D_j D_i^2 B_k)    (repeated indices summed)
//
// Per batch of timeslices: one kernel forms B, three launches of one
// derivative kernel form the 39 derivative fields the operators use (each a
// list of (input field, direction, output field) tasks: D_j B_k; D_j^2 B_k,
// D_j D_k B_j; D_j^3 B_k, D_j^2 D_k B_j, D_j D_i^2 B_k), and a trace kernel
// sums the five traces over the sites (block partials, then a fixed-order
// final sum: deterministic).  Every field is a 3 x 3 complex matrix per
// site in complex128 (144 bytes).  The work is about 45 kflop per site, far
// from any memory bound: FP64 keeps the operators exact to rounding.
#include <math.h>

#include "common.cuh"
#include "prof.cuh"

namespace distil {

namespace {

constexpr int GL_NF = 57;         // field slots per timeslice (see field_* below)
constexpr int GL_MAX_TASKS = 18;  // tasks of one derivative launch
constexpr int GL_TRACE_THREADS = 256;

// field slots: B_i 0..2; D1[j][k] = D_j B_k 3..11; D2[j][k] = D_j^2 B_k
// 12..20; E1[j][k] = D_j D_k B_j 21..29; D3[j][k] = D_j^3 B_k 30..38;
// E2[j][k] = D_j^2 D_k B_j 39..47; G[i][k] = D_j D_i^2 B_k (j the third
// index) 48..56
__host__ __device__ constexpr int f_b(int i) { return i; }
__host__ __device__ constexpr int f_d1(int j, int k) { return 3 + 3 * j + k; }
__host__ __device__ constexpr int f_d2(int j, int k) { return 12 + 3 * j + k; }
__host__ __device__ constexpr int f_e1(int j, int k) { return 21 + 3 * j + k; }
__host__ __device__ constexpr int f_d3(int j, int k) { return 30 + 3 * j + k; }
__host__ __device__ constexpr int f_e2(int j, int k) { return 39 + 3 * j + k; }
__host__ __device__ constexpr int f_g(int i, int k) { return 48 + 3 * i + k; }

struct M3 {
  double2 a[9];
};

__device__ __forceinline__ double2 cfma2(double2 x, double2 y, double2 acc) {
  acc.x = fma(x.x, y.x, acc.x);
  acc.x = fma(-x.y, y.y, acc.x);
  acc.y = fma(x.x, y.y, acc.y);
  acc.y = fma(x.y, y.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cconj2(double2 x) { return make_double2(x.x, -x.y); }

__device__ __forceinline__ M3 load_link(const float2* p) {
  M3 m;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.a[e] = make_double2((double)p[e].x, (double)p[e].y);
  return m;
}
__device__ __forceinline__ M3 load_field(const double2* p) {
  M3 m;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.a[e] = p[e];
  return m;
}
__device__ __forceinline__ void store_field(double2* p, const M3& m) {
#pragma unroll
  for (int e = 0; e < 9; ++e) p[e] = m.a[e];
}
// x y
__device__ __forceinline__ M3 mm(const M3& x, const M3& y) {
  M3 r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < 3; ++c) s = cfma2(x.a[3 * a + c], y.a[3 * c + b], s);
      r.a[3 * a + b] = s;
    }
  return r;
}
// x y^dag
__device__ __forceinline__ M3 mmd(const M3& x, const M3& y) {
  M3 r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < 3; ++c) s = cfma2(x.a[3 * a + c], cconj2(y.a[3 * b + c]), s);
      r.a[3 * a + b] = s;
    }
  return r;
}
// x^dag y
__device__ __forceinline__ M3 mdm(const M3& x, const M3& y) {
  M3 r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < 3; ++c) s = cfma2(cconj2(x.a[3 * c + a]), y.a[3 * c + b], s);
      r.a[3 * a + b] = s;
    }
  return r;
}
// Tr(x y)
__device__ __forceinline__ double2 trmm(const M3& x, const M3& y) {
  double2 s = make_double2(0.0, 0.0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) s = cfma2(x.a[3 * a + c], y.a[3 * c + a], s);
  return s;
}

__device__ __forceinline__ int eps3(int i, int j, int k) {
  return (i == j || j == k || i == k) ? 0 : ((j - i + 3) % 3 == 1 ? 1 : -1);
}

// site s + d0 e_x + d1 e_y + d2 e_z on the periodic L^3 lattice
__device__ __forceinline__ int site_at(const int (&c)[3], int L, int d0, int d1, int d2) {
  const int x = (c[0] + d0 + L) % L, y = (c[1] + d1 + L) % L, z = (c[2] + d2 + L) % L;
  return x + L * (y + L * z);
}
__device__ __forceinline__ int site_dir(const int (&c)[3], int L, int k, int step) {
  return site_at(c, L, k == 0 ? step : 0, k == 1 ? step : 0, k == 2 ? step : 0);
}

}  // namespace

// B_i(x) for the timeslices of a batch: one thread per (u, i, s).
__global__ void __launch_bounds__(128) glue_clover_kernel(const float2* __restrict__ U, int L, int nb,
                                                          double2* __restrict__ fields) {
  const long long V3 = (long long)L * L * L;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nb * 3 * V3) return;
  const int s = (int)(idx % V3);
  const int i = (int)((idx / V3) % 3);
  const long long u = idx / (3 * V3);
  const int mu = (i + 1) % 3, nu = (i + 2) % 3;
  const int c[3] = {s % L, (s / L) % L, s / (L * L)};
  const float2* Um = U + (u * 3 + mu) * V3 * 9;
  const float2* Un = U + (u * 3 + nu) * V3 * 9;
  auto um = [&](int d_mu, int d_nu) {
    int d[3] = {0, 0, 0};
    d[mu] += d_mu;
    d[nu] += d_nu;
    return load_link(Um + (long long)site_at(c, L, d[0], d[1], d[2]) * 9);
  };
  auto un = [&](int d_mu, int d_nu) {
    int d[3] = {0, 0, 0};
    d[mu] += d_mu;
    d[nu] += d_nu;
    return load_link(Un + (long long)site_at(c, L, d[0], d[1], d[2]) * 9);
  };
  // the four counter-clockwise plaquettes of the (mu, nu) plane through x:
  //   U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  //   U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  //   U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  //   U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
  M3 q = mmd(mmd(mm(um(0, 0), un(1, 0)), um(0, 1)), un(0, 0));
  const M3 l2 = mm(mmd(mmd(un(0, 0), um(-1, 1)), un(-1, 0)), um(-1, 0));
  const M3 l3 = mdm(mm(un(-1, -1), um(-1, 0)), mm(um(-1, -1), un(0, -1)));
  const M3 l4 = mmd(mm(mdm(un(0, -1), um(0, -1)), un(1, -1)), um(0, 0));
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    q.a[e].x += l2.a[e].x + l3.a[e].x + l4.a[e].x;
    q.a[e].y += l2.a[e].y + l3.a[e].y + l4.a[e].y;
  }
  // F = (Q - Q^dag) / (8 i), traceless; B = 2 F
  M3 b;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 z = q.a[3 * r + k], w = cconj2(q.a[3 * k + r]);
      const double2 dz = make_double2(z.x - w.x, z.y - w.y);
      b.a[3 * r + k] = make_double2(2.0 * dz.y / 8.0, -2.0 * dz.x / 8.0);  // 2 dz / (8 i)
    }
  const double tr = (b.a[0].x + b.a[4].x + b.a[8].x) / 3.0;  // B is Hermitian: its trace is real
  b.a[0].x -= tr;
  b.a[4].x -= tr;
  b.a[8].x -= tr;
  store_field(fields + ((u * GL_NF + f_b(i)) * V3 + s) * 9, b);
}

struct GlTasks {
  int n;
  int in[GL_MAX_TASKS], dir[GL_MAX_TASKS], out[GL_MAX_TASKS];
};

// out = D_dir in for every task of the launch: one thread per (task, u, s).
__global__ void __launch_bounds__(128) glue_deriv_kernel(const float2* __restrict__ U, int L, int nb, GlTasks tk,
                                                         double2* __restrict__ fields) {
  const long long V3 = (long long)L * L * L;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)tk.n * nb * V3) return;
  const int s = (int)(idx % V3);
  const long long u = (idx / V3) % nb;
  const int t = (int)(idx / (V3 * nb));
  const int j = tk.dir[t];
  const int c[3] = {s % L, (s / L) % L, s / (L * L)};
  const int sp = site_dir(c, L, j, 1), sm = site_dir(c, L, j, -1);
  const float2* Uj = U + (u * 3 + j) * V3 * 9;
  const double2* X = fields + (u * GL_NF + tk.in[t]) * V3 * 9;
  const M3 uf = load_link(Uj + (long long)s * 9), ub = load_link(Uj + (long long)sm * 9);
  const M3 fwd = mmd(mm(uf, load_field(X + (long long)sp * 9)), uf);  // U_j(x) X(x+j) U_j(x)^dag
  const M3 bwd = mm(mdm(ub, load_field(X + (long long)sm * 9)), ub);  // U_j(x-j)^dag X(x-j) U_j(x-j)
  M3 r;
#pragma unroll
  for (int e = 0; e < 9; ++e) r.a[e] = make_double2(0.5 * (fwd.a[e].x - bwd.a[e].x), 0.5 * (fwd.a[e].y - bwd.a[e].y));
  store_field(fields + ((u * GL_NF + tk.out[t]) * V3 + s) * 9, r);
}

// Per-block partial sums of the five traces: block (site chunk, u).
__global__ void __launch_bounds__(GL_TRACE_THREADS) glue_trace_kernel(const double2* __restrict__ fields, int L,
                                                                      double2* __restrict__ part) {
  const long long V3 = (long long)L * L * L;
  const long long u = blockIdx.y;
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double2 o[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) o[n] = make_double2(0.0, 0.0);
  if (s < V3) {
    auto F = [&](int f) { return load_field(fields + ((u * GL_NF + f) * V3 + s) * 9); };
    M3 B[3] = {F(f_b(0)), F(f_b(1)), F(f_b(2))};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          const int e = eps3(i, j, k);
          if (!e) continue;
          const double2 t1 = trmm(B[i], F(f_d1(j, k)));
          const double2 t3 = trmm(B[i], F(f_d3(j, k)));
          const double2 t4 = trmm(B[i], F(f_e2(j, k)));
          const double2 t5 = trmm(B[i], F(f_g(i, k)));
          o[0].x += e * t1.x; o[0].y += e * t1.y;
          o[2].x += e * t3.x; o[2].y += e * t3.y;
          o[3].x += e * t4.x; o[3].y += e * t4.y;
          o[4].x += e * t5.x; o[4].y += e * t5.y;
          // O_2: eps_ijk eps_ilm Tr(B_j B_k D_l B_m), (l, m) the two orders of the other pair
          const M3 bb = mm(B[j], B[k]);
          for (int l = 0; l < 3; ++l)
            for (int m = 0; m < 3; ++m) {
              const int e2 = eps3(i, l, m);
              if (!e2) continue;
              const double2 t2 = trmm(bb, F(f_d1(l, m)));
              o[1].x += e * e2 * t2.x;
              o[1].y += e * e2 * t2.y;
            }
        }
  }
  __shared__ double red[2][5][GL_TRACE_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    double x = o[n].x, y = o[n].y;
    for (int off = 16; off > 0; off >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, off);
      y += __shfl_xor_sync(0xffffffffu, y, off);
    }
    if (lane == 0) {
      red[0][n][w] = x;
      red[1][n][w] = y;
    }
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double x = 0.0, y = 0.0;
    for (int k = 0; k < GL_TRACE_THREADS / 32; ++k) {
      x += red[0][threadIdx.x][k];
      y += red[1][threadIdx.x][k];
    }
    part[(u * gridDim.x + blockIdx.x) * 5 + threadIdx.x] = make_double2(x, y);
  }
}

// O[u][n] = sum of the block partials, in block order
__global__ void glue_final_kernel(const double2* __restrict__ part, int nblk, int nb, double2* __restrict__ O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb * 5) return;
  const int u = e / 5, n = e % 5;
  double x = 0.0, y = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double2 p = part[((long long)u * nblk + b) * 5 + n];
    x += p.x;
    y += p.y;
  }
  O[e] = make_double2(x, y);
}

// Timeslices per batch: the fields of a batch within 4 GiB.
static int glue_batch(int L, int nt) {
  const long long V3 = (long long)L * L * L;
  const long long per = (long long)GL_NF * V3 * 9 * 16;
  long long tb = (4LL << 30) / per;
  if (tb < 1) tb = 1;
  return (int)(tb < nt ? tb : nt);
}

size_t glueball_workspace(int L, int nt) {
  const long long V3 = (long long)L * L * L;
  const int tb = glue_batch(L, nt);
  const long long nblk = (V3 + GL_TRACE_THREADS - 1) / GL_TRACE_THREADS;
  Arena ar;
  ar.take<double2>((size_t)tb * GL_NF * V3 * 9);
  ar.take<double2>((size_t)tb * nblk * 5);
  return ar.used + 256;
}

int glueball_operators(distil_ctx* ctx, const void* Uv, int L, int nt, void* Ov, void* ws, size_t ws_bytes,
                       cudaStream_t s) {
  const long long V3 = (long long)L * L * L;
  const int tb = glue_batch(L, nt);
  const long long nblk = (V3 + GL_TRACE_THREADS - 1) / GL_TRACE_THREADS;
  Arena ar(ws, ws_bytes);
  double2* fields = ar.take<double2>((size_t)tb * GL_NF * V3 * 9);
  double2* part = ar.take<double2>((size_t)tb * nblk * 5);
  if (!ar.fits()) {
    set_error("distil_glueball_operators: workspace too small");
    return DISTIL_ENOMEM;
  }
  // derivative tasks of the three depths
  GlTasks st[3] = {};
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      GlTasks& a = st[0];
      a.in[a.n] = f_b(k), a.dir[a.n] = j, a.out[a.n] = f_d1(j, k), ++a.n;  // D_j B_k
      if (j == k) continue;
      GlTasks& b = st[1];
      b.in[b.n] = f_d1(j, k), b.dir[b.n] = j, b.out[b.n] = f_d2(j, k), ++b.n;  // D_j^2 B_k
      b.in[b.n] = f_d1(k, j), b.dir[b.n] = j, b.out[b.n] = f_e1(j, k), ++b.n;  // D_j D_k B_j
      GlTasks& c = st[2];
      c.in[c.n] = f_d2(j, k), c.dir[c.n] = j, c.out[c.n] = f_d3(j, k), ++c.n;  // D_j^3 B_k
      c.in[c.n] = f_e1(j, k), c.dir[c.n] = j, c.out[c.n] = f_e2(j, k), ++c.n;  // D_j^2 D_k B_j
    }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      if (i == k) continue;
      const int j = 3 - i - k;  // the third index
      GlTasks& c = st[2];
      c.in[c.n] = f_d2(i, k), c.dir[c.n] = j, c.out[c.n] = f_g(i, k), ++c.n;  // D_j D_i^2 B_k
    }
  for (int t0 = 0; t0 < nt; t0 += tb) {
    const int nb = nt - t0 < tb ? nt - t0 : tb;
    const float2* U = reinterpret_cast<const float2*>(Uv) + (long long)t0 * 3 * V3 * 9;
    {
      Launch Lc(ctx, "glue_clover", s);
      const long long n = (long long)nb * 3 * V3;
      glue_clover_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(U, L, nb, fields);
    }
    DISTIL_LAUNCH_CHECK();
    for (int d = 0; d < 3; ++d) {
      Launch Ld(ctx, "glue_deriv", s);
      const long long n = (long long)st[d].n * nb * V3;
      glue_deriv_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(U, L, nb, st[d], fields);
      DISTIL_LAUNCH_CHECK();
    }
    {
      Launch Lt(ctx, "glue_trace", s);
      glue_trace_kernel<<<dim3((unsigned)nblk, (unsigned)nb), GL_TRACE_THREADS, 0, s>>>(fields, L, part);
      glue_final_kernel<<<(nb * 5 + 127) / 128, 128, 0, s>>>(part, (int)nblk, nb,
                                                             reinterpret_cast<double2*>(Ov) + (long long)t0 * 5);
    }
    DISTIL_LAUNCH_CHECK();
  }
  return DISTIL_OK;
}

}  // namespace distil
