// Generalized eigenvalues (and optionally eigenvectors) of the N_B x N_B
// correlation matrices (Sec. 2.1: "compute an N_B x N_B correlation matrix
// and solve a GEVP"), FP64.
//
// For each (q, t): M = C(t0)^{-1} C(t) by Gaussian elimination with partial
// pivoting, Householder reduction of M to upper Hessenberg form, then
// explicitly shifted complex QR sweeps (Wilkinson shift, exceptional shift
// every 10 stalled sweeps) with deflation at negligible subdiagonals.  When
// eigenvectors are wanted the reflections and rotations are applied to the
// whole matrix and accumulated in Z, so that M = Z T Z^H with T upper
// triangular (complex Schur form); the eigenvector of T for its j-th
// diagonal entry follows by back substitution and is mapped back by Z.
// Eigenvalues are sorted by |lambda| descending (stable); each eigenvector
// is scaled to unit 2-norm and its largest-modulus component made real and
// positive.  One thread per problem; N_B <= 16 keeps the matrices in
// thread-local storage.
#include "common.cuh"
#include "prof.cuh"

namespace distil {

constexpr int GV_MAX = 16;

__device__ __forceinline__ double cabs_(Cx<double> z) { return hypot(z.r, z.i); }
__device__ __forceinline__ Cx<double> cdiv_(Cx<double> a, Cx<double> b) {
  // Smith's algorithm
  if (fabs(b.r) >= fabs(b.i)) {
    double r = b.i / b.r, d = b.r + b.i * r;
    return cmake((a.r + a.i * r) / d, (a.i - a.r * r) / d);
  } else {
    double r = b.r / b.i, d = b.r * r + b.i;
    return cmake((a.r * r + a.i) / d, (a.i * r - a.r) / d);
  }
}
__device__ __forceinline__ Cx<double> csqrt_(Cx<double> z) {
  double m = cabs_(z);
  if (m == 0.0) return cmake(0.0, 0.0);
  double re = sqrt(0.5 * (m + fabs(z.r)));
  double im = 0.5 * z.i / re;
  if (z.r >= 0) return cmake(re, im);
  return cmake(fabs(im), z.i >= 0 ? re : -re);
}

__global__ void gevp_kernel(const Cx<double>* __restrict__ C, int np, int nb, int nt, int t0, int t_begin,
                            int t_count, Cx<double>* __restrict__ lam, Cx<double>* __restrict__ vecs) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= np * t_count) return;
  const int q = id / t_count, t = t_begin + id % t_count;
  const bool want = vecs != nullptr;
  Cx<double> A[GV_MAX][GV_MAX], H[GV_MAX][GV_MAX], Z[GV_MAX][GV_MAX];
  const int n = nb;
  const Cx<double>* Cq = C + (long long)q * nb * nb * nt;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      A[a][b] = Cq[((long long)a * nb + b) * nt + t0];
      H[a][b] = Cq[((long long)a * nb + b) * nt + t];
      Z[a][b] = cmake(a == b ? 1.0 : 0.0, 0.0);
    }
  Cx<double>* out = lam + ((long long)q * nt + t) * nb;
  Cx<double>* vout = want ? vecs + ((long long)q * nt + t) * nb * nb : nullptr;
  const Cx<double> nanv = cmake(nan(""), nan(""));
  auto fail = [&]() {
    for (int a = 0; a < n; ++a) out[a] = nanv;
    if (want)
      for (int a = 0; a < n * n; ++a) vout[a] = nanv;
  };
  // ---- solve A M = H in place (H <- M), partial pivoting
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = cabs_(A[c][c]);
    for (int r = c + 1; r < n; ++r)
      if (cabs_(A[r][c]) > best) { best = cabs_(A[r][c]); piv = r; }
    if (!(best > 0.0)) {
      fail();
      return;
    }
    if (piv != c) {
      for (int b = 0; b < n; ++b) {
        Cx<double> tmp = A[c][b]; A[c][b] = A[piv][b]; A[piv][b] = tmp;
        tmp = H[c][b]; H[c][b] = H[piv][b]; H[piv][b] = tmp;
      }
    }
    for (int r = c + 1; r < n; ++r) {
      Cx<double> f = cdiv_(A[r][c], A[c][c]);
      for (int b = c; b < n; ++b) A[r][b] = csub(A[r][b], cmul(f, A[c][b]));
      for (int b = 0; b < n; ++b) H[r][b] = csub(H[r][b], cmul(f, H[c][b]));
    }
  }
  for (int c = n - 1; c >= 0; --c)
    for (int b = 0; b < n; ++b) {
      Cx<double> s = H[c][b];
      for (int k = c + 1; k < n; ++k) s = csub(s, cmul(A[c][k], H[k][b]));
      H[c][b] = cdiv_(s, A[c][c]);
    }
  // ---- Householder reduction to Hessenberg form, H <- P H P, Z <- Z P
  for (int k = 0; k < n - 2; ++k) {
    double alpha = 0;
    for (int r = k + 1; r < n; ++r) alpha += H[r][k].r * H[r][k].r + H[r][k].i * H[r][k].i;
    alpha = sqrt(alpha);
    if (alpha == 0.0) continue;
    Cx<double> x0 = H[k + 1][k];
    double ax0 = cabs_(x0);
    Cx<double> ph = ax0 > 0 ? cscale(x0, 1.0 / ax0) : cmake(1.0, 0.0);
    Cx<double> u[GV_MAX];
    for (int r = 0; r < n; ++r) u[r] = cmake(0.0, 0.0);
    u[k + 1] = cadd(x0, cscale(ph, alpha));
    for (int r = k + 2; r < n; ++r) u[r] = H[r][k];
    double un = 0;
    for (int r = k + 1; r < n; ++r) un += u[r].r * u[r].r + u[r].i * u[r].i;
    if (un == 0.0) continue;
    double beta = 2.0 / un;
    // H <- (I - beta u u^H) H
    for (int b = 0; b < n; ++b) {
      Cx<double> s = cmake(0.0, 0.0);
      for (int r = k + 1; r < n; ++r) s = cadd(s, cmul(cconj(u[r]), H[r][b]));
      s = cscale(s, beta);
      for (int r = k + 1; r < n; ++r) H[r][b] = csub(H[r][b], cmul(u[r], s));
    }
    // H <- H (I - beta u u^H), and the same for Z
    for (int a = 0; a < n; ++a) {
      Cx<double> s = cmake(0.0, 0.0);
      for (int r = k + 1; r < n; ++r) s = cadd(s, cmul(H[a][r], u[r]));
      s = cscale(s, beta);
      for (int r = k + 1; r < n; ++r) H[a][r] = csub(H[a][r], cmul(s, cconj(u[r])));
    }
    if (want)
      for (int a = 0; a < n; ++a) {
        Cx<double> s = cmake(0.0, 0.0);
        for (int r = k + 1; r < n; ++r) s = cadd(s, cmul(Z[a][r], u[r]));
        s = cscale(s, beta);
        for (int r = k + 1; r < n; ++r) Z[a][r] = csub(Z[a][r], cmul(s, cconj(u[r])));
      }
    for (int r = k + 2; r < n; ++r) H[r][k] = cmake(0.0, 0.0);
  }
  // ---- shifted QR on the active window [l, hi]; with eigenvectors the
  // rotations act on the whole rows / columns (full Schur form)
  int hi = n - 1, stall = 0, total = 0;
  const double eps = 2.220446049250313e-16;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double sub = cabs_(H[l][l - 1]);
      double dia = cabs_(H[l - 1][l - 1]) + cabs_(H[l][l]);
      if (sub <= eps * dia || sub < 1e-300) { H[l][l - 1] = cmake(0.0, 0.0); break; }
      --l;
    }
    if (l == hi) { --hi; stall = 0; continue; }
    if (++total > 60 * n) {
      fail();
      return;
    }
    Cx<double> mu;
    if (++stall % 11 == 10) {
      mu = cadd(H[hi][hi], cmake(cabs_(H[hi][hi - 1]), 0.0));
    } else {
      Cx<double> a = H[hi - 1][hi - 1], b = H[hi - 1][hi], c = H[hi][hi - 1], d = H[hi][hi];
      Cx<double> half = cscale(csub(a, d), 0.5);
      Cx<double> disc = csqrt_(cadd(cmul(half, half), cmul(b, c)));
      Cx<double> m1 = cadd(cscale(cadd(a, d), 0.5), disc), m2 = csub(cscale(cadd(a, d), 0.5), disc);
      mu = (cabs_(csub(m1, d)) <= cabs_(csub(m2, d))) ? m1 : m2;
    }
    for (int k = l; k <= hi; ++k) H[k][k] = csub(H[k][k], mu);
    double gc[GV_MAX];
    Cx<double> gs[GV_MAX];
    const int bend = want ? n - 1 : hi;
    for (int k = l; k < hi; ++k) {
      Cx<double> a = H[k][k], b = H[k + 1][k];
      double aa = cabs_(a), bb = cabs_(b);
      double c;
      Cx<double> s;
      if (bb == 0.0) { c = 1.0; s = cmake(0.0, 0.0); }
      else if (aa == 0.0) { c = 0.0; s = cmake(1.0, 0.0); }
      else {
        double r = hypot(aa, bb);
        c = aa / r;
        s = cscale(cmul(cscale(a, 1.0 / aa), cconj(b)), 1.0 / r);
      }
      gc[k] = c; gs[k] = s;
      for (int b2 = k; b2 <= bend; ++b2) {
        Cx<double> x = H[k][b2], y = H[k + 1][b2];
        H[k][b2] = cadd(cscale(x, c), cmul(s, y));
        H[k + 1][b2] = csub(cscale(y, c), cmul(cconj(s), x));
      }
    }
    const int abegin = want ? 0 : l;
    for (int k = l; k < hi; ++k) {
      double c = gc[k];
      Cx<double> s = gs[k];
      int rmax = (k + 2 < hi) ? k + 2 : hi;
      for (int a = abegin; a <= rmax; ++a) {
        Cx<double> x = H[a][k], y = H[a][k + 1];
        H[a][k] = cadd(cscale(x, c), cmul(y, cconj(s)));
        H[a][k + 1] = csub(cscale(y, c), cmul(x, s));
      }
      if (want)
        for (int a = 0; a < n; ++a) {
          Cx<double> x = Z[a][k], y = Z[a][k + 1];
          Z[a][k] = cadd(cscale(x, c), cmul(y, cconj(s)));
          Z[a][k + 1] = csub(cscale(y, c), cmul(x, s));
        }
    }
    for (int k = l; k <= hi; ++k) H[k][k] = cadd(H[k][k], mu);
  }
  // ---- sort by modulus, largest first (stable insertion sort of indices)
  int order[GV_MAX];
  for (int a = 0; a < n; ++a) order[a] = a;
  for (int a = 1; a < n; ++a) {
    const int key = order[a];
    const double km = cabs_(H[key][key]);
    int b = a - 1;
    while (b >= 0 && cabs_(H[order[b]][order[b]]) < km) { order[b + 1] = order[b]; --b; }
    order[b + 1] = key;
  }
  for (int a = 0; a < n; ++a) out[a] = H[order[a]][order[a]];
  if (!want) return;
  // ---- eigenvectors: T y = T_jj y by back substitution, x = Z y
  double tnorm = 0.0;
  for (int a = 0; a < n; ++a)
    for (int b = a; b < n; ++b) tnorm = fmax(tnorm, cabs_(H[a][b]));
  const double small = fmax(eps * tnorm, 1e-300);
  for (int m = 0; m < n; ++m) {
    const int j = order[m];
    Cx<double> y[GV_MAX];
    for (int i = 0; i < n; ++i) y[i] = cmake(i == j ? 1.0 : 0.0, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      Cx<double> s = cmake(0.0, 0.0);
      for (int k = i + 1; k <= j; ++k) s = cadd(s, cmul(H[i][k], y[k]));
      Cx<double> d = csub(H[i][i], H[j][j]);
      if (cabs_(d) < small) d = cmake(small, 0.0);
      y[i] = cscale(cdiv_(s, d), -1.0);
    }
    Cx<double> x[GV_MAX];
    double nrm = 0.0, big = -1.0;
    int ibig = 0;
    for (int a = 0; a < n; ++a) {
      Cx<double> acc = cmake(0.0, 0.0);
      for (int k = 0; k <= j; ++k) acc = cadd(acc, cmul(Z[a][k], y[k]));
      x[a] = acc;
      const double m2 = acc.r * acc.r + acc.i * acc.i;
      nrm += m2;
      if (m2 > big) { big = m2; ibig = a; }
    }
    // unit norm, largest component real and positive
    const double ab = sqrt(big);
    const Cx<double> ph = ab > 0 ? cscale(cconj(x[ibig]), 1.0 / (ab * sqrt(nrm))) : cmake(0.0, 0.0);
    for (int a = 0; a < n; ++a) vout[(long long)m * nb + a] = cmul(x[a], ph);
  }
}

// Correlators of the optimal operators: copt[q][n][t] = u^H C(t) u with u =
// vecs[q][td][n][:] (a GEVP eigenvector), and the effective masses
// meff[q][n][t] = log(|copt(t)| / |copt(t+1)|), NaN at the last timeslice.
// One thread per (q, n).
__global__ void optimal_kernel(const Cx<double>* __restrict__ C, int np, int nb, int nt,
                               const Cx<double>* __restrict__ vecs, int td, Cx<double>* __restrict__ copt,
                               double* __restrict__ meff) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= np * nb) return;
  const int q = id / nb, n = id % nb;
  const Cx<double>* u = vecs + (((long long)q * nt + td) * nb + n) * nb;
  const Cx<double>* Cq = C + (long long)q * nb * nb * nt;
  double prev = 0.0;
  for (int t = 0; t < nt; ++t) {
    Cx<double> acc = cmake(0.0, 0.0);
    for (int a = 0; a < nb; ++a) {
      Cx<double> row = cmake(0.0, 0.0);
      for (int b = 0; b < nb; ++b) row = cadd(row, cmul(Cq[((long long)a * nb + b) * nt + t], u[b]));
      acc = cadd(acc, cmul(cconj(u[a]), row));
    }
    copt[((long long)q * nb + n) * nt + t] = acc;
    const double m = cabs_(acc);
    if (meff && t > 0) meff[((long long)q * nb + n) * nt + t - 1] = log(prev / m);
    prev = m;
  }
  if (meff) meff[((long long)q * nb + n) * nt + nt - 1] = nan("");
}

int optimal_launch(distil_ctx* ctx, const void* C, int np, int nb, int nt, const void* vecs, int td, void* copt,
                   double* meff, cudaStream_t s) {
  const int total = np * nb;
  {
    Launch L(ctx, "optimal", s);
    optimal_kernel<<<(total + 63) / 64, 64, 0, s>>>((const Cx<double>*)C, np, nb, nt, (const Cx<double>*)vecs, td,
                                                    (Cx<double>*)copt, meff);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

// Profiles as Gaussians in the Laplacian eigenvalue: prof[t][b][i] =
// exp(-(lam[t][i] / sigma_b)^2), FP64 (the paper's profiles "can be a
// function of the 3D Laplacian eigenvalues", Sec. 2.1).  The N_B <= 16
// widths travel in the kernel arguments.
struct ProfileWidths {
  double sigma[16];
};
__global__ void eigen_profiles_kernel(const double* __restrict__ lam, int nt, int nv, ProfileWidths w, int nb,
                                      double* __restrict__ prof) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)nt * nb * nv;
  if (e >= total) return;
  const int i = (int)(e % nv);
  const long long tb = e / nv;
  const int b = (int)(tb % nb), t = (int)(tb / nb);
  const double x = lam[(long long)t * nv + i] / w.sigma[b];
  prof[e] = exp(-x * x);
}

int eigen_profiles_launch(distil_ctx* ctx, const double* lam, int nt, int nv, const double* sigma, int nb,
                          double* prof, cudaStream_t s) {
  ProfileWidths w{};
  for (int b = 0; b < nb && b < 16; ++b) w.sigma[b] = sigma[b];
  const long long total = (long long)nt * nb * nv;
  {
    Launch L(ctx, "eigen_profiles", s);
    eigen_profiles_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(lam, nt, nv, w, nb, prof);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

int gevp_launch(distil_ctx* ctx, const void* C, int np, int nb, int nt, int t0, int t_begin, int t_count,
                void* lambda, void* vecs, cudaStream_t s) {
  int total = np * t_count;
  if (total == 0) return DISTIL_OK;
  {
    Launch L(ctx, "gevp", s);
    gevp_kernel<<<(total + 63) / 64, 64, 0, s>>>((const Cx<double>*)C, np, nb, nt, t0, t_begin, t_count,
                                                 (Cx<double>*)lambda, (Cx<double>*)vecs);
  }
  DISTIL_LAUNCH_CHECK();
  return DISTIL_OK;
}

}  // namespace distil
