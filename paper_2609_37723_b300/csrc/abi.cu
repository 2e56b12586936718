// C-ABI entry points of libdistil (declared in include/distil.h): argument
// validation, workspace accounting and dispatch to the kernels of each mode.
#include <stdint.h>
#include <stdarg.h>
#include <string.h>

#include "common.cuh"
#include "correlate.cuh"
#include "elementals.cuh"
#include "mixed.cuh"
#include "prof.cuh"

namespace distil {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* get_error() { return g_err; }

int gevp_launch(distil_ctx* ctx, const void* C, int np, int nb, int nt, int t0, int t_begin, int t_count,
                void* lambda, void* vecs, cudaStream_t s);
int optimal_launch(distil_ctx* ctx, const void* C, int np, int nb, int nt, const void* vecs, int td, void* copt,
                   double* meff, cudaStream_t s);
int eigen_profiles_launch(distil_ctx* ctx, const double* lam, int nt, int nv, const double* sigma, int nb,
                          double* prof, cudaStream_t s);

size_t meson_elementals_workspace(int L, int nt, int nv, int np);
int meson_elementals(distil_ctx* ctx, const void* v, const void* U, int L, int nt, int nv, const int32_t* mom,
                     int np, void* phi, void* ws, size_t ws_bytes, cudaStream_t s);
size_t meson_correlate_workspace(int nv, int np, int nb);
int meson_correlate(distil_ctx* ctx, const void* phi_snk, const void* phi_src, const void* tau, int nt, int nv,
                    int np, const double* prof, int nb, void* C, void* ws, size_t ws_bytes, cudaStream_t s);
int meson_prune(distil_ctx* ctx, const void* C, int np, int nops, int nt, int tp, int nkeep, void* Ct, void* Un,
                double* sv, cudaStream_t s);

size_t glueball_workspace(int L, int nt);
int glueball_operators(distil_ctx* ctx, const void* U, int L, int nt, void* O, void* ws, size_t ws_bytes,
                       cudaStream_t s);

Profiler& profiler(distil_ctx* ctx) { return *ctx->prof; }

// Lowest index of a NaN or Inf among x[0, count) into the 64-bit word *slot
// (which starts at LLONG_MAX).
__global__ void scan_finite_kernel(const void* __restrict__ x, long long count, int f32,
                                   unsigned long long* __restrict__ slot) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const bool fin = f32 ? isfinite(static_cast<const float*>(x)[i]) : isfinite(static_cast<const double*>(x)[i]);
    if (!fin) atomicMin(slot, (unsigned long long)i);
  }
}

// Synchronous on `s`: *bad = the first non-finite element or -1.  The scan
// uses the spare 64-bit word of the context's device status buffer.
int scan_finite_launch(distil_ctx* ctx, const void* x, long long count, bool f32, long long* bad, cudaStream_t s) {
  unsigned long long* slot = reinterpret_cast<unsigned long long*>(ctx->d_error + 2);
  const unsigned long long init = ~0ull;
  DISTIL_CUDA(cudaMemcpyAsync(slot, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  if (count > 0) {
    Launch L(ctx, "scan_finite", s);
    long long blocks = (count + 255) / 256;
    if (blocks > 4 * 148 * 8) blocks = 4 * 148 * 8;
    scan_finite_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, count, f32 ? 1 : 0, slot);
  }
  DISTIL_LAUNCH_CHECK();
  unsigned long long got = 0;
  DISTIL_CUDA(cudaMemcpyAsync(&got, slot, sizeof(got), cudaMemcpyDeviceToHost, s));
  DISTIL_CUDA(cudaStreamSynchronize(s));
  *bad = got == ~0ull ? -1 : (long long)got;
  return DISTIL_OK;
}

// Make the context's device current for this call.
static int enter(distil_ctx* ctx) {
  if (!ctx) {
    set_error("null context");
    return DISTIL_EINVAL;
  }
  DISTIL_CUDA(cudaSetDevice(ctx->device));
  return DISTIL_OK;
}

}  // namespace distil

using namespace distil;

extern "C" {

int distil_create(int device, distil_ctx** out) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(out != nullptr, "distil_create: out is null");
  *out = nullptr;
  int ndev = 0;
  DISTIL_CUDA(cudaGetDeviceCount(&ndev));
  DISTIL_CHECK_ARG(device >= 0 && device < ndev, "distil_create: device %d not in [0,%d)", device, ndev);
  DISTIL_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  DISTIL_CUDA(cudaGetDeviceProperties(&prop, device));
  distil_ctx* c = new distil_ctx();
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  c->cc_major = prop.major;
  c->cc_minor = prop.minor;
  c->d_error = nullptr;
  c->prof = new Profiler();
  // every site: persistent CTAs with one accumulator set of the widest tile
  // (128 wide at step i, 80 / 64 with three pairs), the copies of the next
  // tile running during the epilogue (measured fastest at N_v = 256)
  c->tune[0] = 5;  // step i (K = N_v)
  c->tune[1] = 5;  // step j (K = 4 N_v)
  c->tune[2] = 5;  // T contraction (K = 5 N_v)
  c->wait_limit = 0;
  if (cudaMalloc(&c->d_error, sizeof(unsigned int) * 4) != cudaSuccess ||
      cudaMemset(c->d_error, 0, sizeof(unsigned int) * 4) != cudaSuccess) {
    set_error("distil_create: cannot allocate the device error word");
    delete c->prof;
    delete c;
    return DISTIL_ENOMEM;
  }
  *out = c;
  return DISTIL_OK;
}

void distil_destroy(distil_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->d_error) cudaFree(ctx->d_error);
  delete ctx->prof;
  delete ctx;
}

const char* distil_last_error(void) { return get_error(); }

int distil_elementals_workspace(int L, int nt, int nv, int np, int mode, size_t* bytes) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(bytes != nullptr, "bytes is null");
  DISTIL_CHECK_ARG(valid_mode(mode), "bad mode %d", mode);
  DISTIL_CHECK_ARG(L >= 1 && nt >= 1 && nv >= 1 && np >= 1, "bad sizes");
  *bytes = is_mixed(mode) ? elementals_mixed_workspace(L, nt, nv, np, mode) : 0;
  return DISTIL_OK;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int distil_elementals(distil_ctx* ctx, const void* v, int L, int nt, int nv, const int32_t* mom, int np,
                      int mode, void* phi, void* workspace, size_t ws_bytes, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(valid_mode(mode), "distil_elementals: bad mode %d", mode);
  DISTIL_CHECK_ARG(L >= 1 && L <= EL_MAX_L, "distil_elementals: L=%d outside [1,%d]", L, EL_MAX_L);
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && np >= 1, "distil_elementals: nt, nv, np must be >= 1");
  DISTIL_CHECK_ARG(np <= EL_MAX_MOM, "distil_elementals: at most %d momenta per call", EL_MAX_MOM);
  DISTIL_CHECK_ARG(mom && ((v && phi) || comb3(nv) == 0), "distil_elementals: null pointer");
  DISTIL_CHECK_ARG(aligned(v, mode == DISTIL_FP64 ? 16 : 8) && aligned(phi, mode == DISTIL_FP32 ? 8 : 16) &&
                       aligned(workspace, 256),
                   "distil_elementals: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == DISTIL_FP64)
    return elementals_simt<double>(ctx, (const Cx<double>*)v, L, nt, nv, mom, np, (Cx<double>*)phi, s);
  if (mode == DISTIL_FP32)
    return elementals_simt<float>(ctx, (const Cx<float>*)v, L, nt, nv, mom, np, (Cx<float>*)phi, s);
  size_t need = elementals_mixed_workspace(L, nt, nv, np, mode);
  if (ws_bytes < need || (need && !workspace)) {
    set_error("distil_elementals: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  return elementals_mixed(ctx, (const Cx<float>*)v, L, nt, nv, mom, np, mode, phi, workspace, ws_bytes, s);
}

int distil_correlate_workspace(int nt, int nv, int np, int nb, int mode, size_t* bytes) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(bytes != nullptr, "bytes is null");
  DISTIL_CHECK_ARG(valid_mode(mode), "bad mode %d", mode);
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && np >= 1 && nb >= 1 && nb <= 16, "bad sizes");
  if (is_mixed(mode)) *bytes = correlate_mixed_workspace(mode, nt, nv, np, nb);
  else *bytes = correlate_plain_workspace(mode == DISTIL_FP64, nv, nb);
  return DISTIL_OK;
}

int distil_correlate(distil_ctx* ctx, const void* phi_snk, const void* phi_src, const void* tau, int nt, int nv,
                     int np, const double* prof, int nb, int prof_per_t, int mode, void* C, void* workspace,
                     size_t ws_bytes, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(valid_mode(mode), "distil_correlate: bad mode %d", mode);
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && np >= 1, "distil_correlate: nt, nv, np must be >= 1");
  DISTIL_CHECK_ARG(nb >= 1 && nb <= 16, "distil_correlate: nb=%d outside [1,16]", nb);
  DISTIL_CHECK_ARG(tau && prof && C && ((phi_snk && phi_src) || comb3(nv) == 0),
                   "distil_correlate: null pointer");
  DISTIL_CHECK_ARG(aligned(phi_snk, mode == DISTIL_FP32 ? 8 : 16) && aligned(phi_src, mode == DISTIL_FP32 ? 8 : 16) &&
                       aligned(tau, mode == DISTIL_FP64 ? 16 : 8) && aligned(prof, 8) && aligned(C, 16) &&
                       aligned(workspace, 256),
                   "distil_correlate: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t need = 0;
  distil_correlate_workspace(nt, nv, np, nb, mode, &need);
  if (nv >= 3 && (ws_bytes < need || !workspace)) {
    set_error("distil_correlate: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  if (is_mixed(mode))
    return correlate_mixed(ctx, mode, phi_snk, phi_src, tau, nt, nv, np, prof, prof, prof_per_t, nb, C, nt, 0,
                           workspace, ws_bytes, s);
  return correlate_plain(ctx, mode == DISTIL_FP64, phi_snk, phi_src, tau, nt, nv, np, prof, prof, prof_per_t, nb, C,
                         nt, 0, workspace, ws_bytes, s);
}

int distil_correlate_slice(distil_ctx* ctx, const void* phi_snk_t, const void* phi_src, const void* tau_t, int nv,
                           int np, const double* prof_snk, const double* prof_src, int nb, int mode, void* C, int nt,
                           int t, void* workspace, size_t ws_bytes, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(valid_mode(mode), "distil_correlate_slice: bad mode %d", mode);
  DISTIL_CHECK_ARG(nv >= 1 && np >= 1 && nt >= 1, "distil_correlate_slice: nv, np, nt must be >= 1");
  DISTIL_CHECK_ARG(t >= 0 && t < nt, "distil_correlate_slice: t=%d outside [0,%d)", t, nt);
  DISTIL_CHECK_ARG(nb >= 1 && nb <= 16, "distil_correlate_slice: nb=%d outside [1,16]", nb);
  DISTIL_CHECK_ARG(tau_t && prof_snk && prof_src && C && ((phi_snk_t && phi_src) || comb3(nv) == 0),
                   "distil_correlate_slice: null pointer");
  const size_t phi_al = mode == DISTIL_FP32 ? 8 : 16;
  DISTIL_CHECK_ARG(aligned(phi_snk_t, phi_al) && aligned(phi_src, phi_al) &&
                       aligned(tau_t, mode == DISTIL_FP64 ? 16 : 8) && aligned(prof_snk, 8) &&
                       aligned(prof_src, 8) && aligned(C, 16) && aligned(workspace, 256),
                   "distil_correlate_slice: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t need = 0;
  distil_correlate_workspace(1, nv, np, nb, mode, &need);
  if (nv >= 3 && (ws_bytes < need || !workspace)) {
    set_error("distil_correlate_slice: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  if (is_mixed(mode))
    return correlate_mixed(ctx, mode, phi_snk_t, phi_src, tau_t, 1, nv, np, prof_snk, prof_src, 0, nb, C, nt, t,
                           workspace, ws_bytes, s);
  return correlate_plain(ctx, mode == DISTIL_FP64, phi_snk_t, phi_src, tau_t, 1, nv, np, prof_snk, prof_src, 0, nb,
                         C, nt, t, workspace, ws_bytes, s);
}

int distil_gevp(distil_ctx* ctx, const void* C, int np, int nb, int nt, int t0, void* lambda,
                distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(C && lambda, "distil_gevp: null pointer");
  DISTIL_CHECK_ARG(np >= 1 && nt >= 1, "distil_gevp: np, nt must be >= 1");
  DISTIL_CHECK_ARG(nb >= 1 && nb <= 16, "distil_gevp: nb=%d outside [1,16]", nb);
  DISTIL_CHECK_ARG(t0 >= 0 && t0 < nt, "distil_gevp: t0=%d outside [0,%d)", t0, nt);
  DISTIL_CHECK_ARG(aligned(C, 16) && aligned(lambda, 16), "distil_gevp: misaligned pointer");
  return gevp_launch(ctx, C, np, nb, nt, t0, 0, nt, lambda, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

int distil_gevp_range(distil_ctx* ctx, const void* C, int np, int nb, int nt, int t0, int t_begin, int t_count,
                      void* lambda, void* vecs, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(C && lambda, "distil_gevp_range: null pointer");
  DISTIL_CHECK_ARG(np >= 1 && nt >= 1, "distil_gevp_range: np, nt must be >= 1");
  DISTIL_CHECK_ARG(nb >= 1 && nb <= 16, "distil_gevp_range: nb=%d outside [1,16]", nb);
  DISTIL_CHECK_ARG(t0 >= 0 && t0 < nt, "distil_gevp_range: t0=%d outside [0,%d)", t0, nt);
  DISTIL_CHECK_ARG(t_begin >= 0 && t_count >= 0 && t_begin + t_count <= nt,
                   "distil_gevp_range: timeslices [%d,%d) outside [0,%d)", t_begin, t_begin + t_count, nt);
  DISTIL_CHECK_ARG(aligned(C, 16) && aligned(lambda, 16) && aligned(vecs, 16), "distil_gevp_range: misaligned pointer");
  return gevp_launch(ctx, C, np, nb, nt, t0, t_begin, t_count, lambda, vecs, reinterpret_cast<cudaStream_t>(stream));
}

int distil_optimal(distil_ctx* ctx, const void* C, int np, int nb, int nt, const void* vecs, int td, void* copt,
                   double* meff, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(C && vecs && copt, "distil_optimal: null pointer");
  DISTIL_CHECK_ARG(np >= 1 && nt >= 1, "distil_optimal: np, nt must be >= 1");
  DISTIL_CHECK_ARG(nb >= 1 && nb <= 16, "distil_optimal: nb=%d outside [1,16]", nb);
  DISTIL_CHECK_ARG(td >= 0 && td < nt, "distil_optimal: td=%d outside [0,%d)", td, nt);
  DISTIL_CHECK_ARG(aligned(C, 16) && aligned(vecs, 16) && aligned(copt, 16) && aligned(meff, 8),
                   "distil_optimal: misaligned pointer");
  return optimal_launch(ctx, C, np, nb, nt, vecs, td, copt, meff, reinterpret_cast<cudaStream_t>(stream));
}

int distil_cgemm_workspace(int M, int N, int K, int batch, int mode, size_t* bytes) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(bytes != nullptr, "bytes is null");
  DISTIL_CHECK_ARG(is_mixed(mode), "distil_cgemm: mode %d is not a tensor-core mode", mode);
  DISTIL_CHECK_ARG(M >= 1 && N >= 1 && K >= 1 && batch >= 1, "bad sizes");
  *bytes = cgemm_workspace(mode, M, N, K, batch);
  return DISTIL_OK;
}

int distil_cgemm(distil_ctx* ctx, const void* A, const void* B, void* C, int M, int N, int K, int batch, int mode,
                 void* workspace, size_t ws_bytes, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(is_mixed(mode), "distil_cgemm: mode %d is not a tensor-core mode", mode);
  DISTIL_CHECK_ARG(M >= 1 && N >= 1 && K >= 1 && batch >= 1 && batch <= 65535, "distil_cgemm: bad sizes");
  DISTIL_CHECK_ARG(A && B && C && workspace, "distil_cgemm: null pointer");
  DISTIL_CHECK_ARG(aligned(A, 8) && aligned(B, 8) && aligned(C, 8) && aligned(workspace, 256),
                   "distil_cgemm: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  size_t need = cgemm_workspace(mode, M, N, K, batch);
  if (ws_bytes < need) {
    set_error("distil_cgemm: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  return cgemm_mixed(ctx, mode, A, B, C, M, N, K, batch, workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ meson path

static constexpr int MS_LIMIT_MOM = 16, MS_LIMIT_NB = 10, MS_LIMIT_NV = 1024, MS_LIMIT_L = 128;

int distil_meson_elementals_workspace(int L, int nt, int nv, int np, int mode, size_t* bytes) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(bytes != nullptr, "bytes is null");
  if (mode != DISTIL_MIXED_FP16X6) {
    set_error("distil_meson_elementals_workspace: mode %d not supported (FP16X6 only)", mode);
    return DISTIL_ENOTSUP;
  }
  DISTIL_CHECK_ARG(L >= 1 && L <= MS_LIMIT_L && nt >= 1 && nv >= 1 && nv <= MS_LIMIT_NV && np >= 1 &&
                       np <= MS_LIMIT_MOM,
                   "distil_meson_elementals_workspace: bad sizes");
  *bytes = meson_elementals_workspace(L, nt, nv, np);
  return DISTIL_OK;
}

int distil_meson_elementals(distil_ctx* ctx, const void* v, const void* U, int L, int nt, int nv,
                            const int32_t* mom, int np, int mode, void* phi, void* workspace, size_t ws_bytes,
                            distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  if (mode != DISTIL_MIXED_FP16X6) {
    set_error("distil_meson_elementals: mode %d not supported (FP16X6 only)", mode);
    return DISTIL_ENOTSUP;
  }
  DISTIL_CHECK_ARG(L >= 1 && L <= MS_LIMIT_L, "distil_meson_elementals: L=%d outside [1,%d]", L, MS_LIMIT_L);
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && nv <= MS_LIMIT_NV, "distil_meson_elementals: nt >= 1, 1 <= nv <= %d",
                   MS_LIMIT_NV);
  DISTIL_CHECK_ARG(np >= 1 && np <= MS_LIMIT_MOM, "distil_meson_elementals: 1 <= np <= %d", MS_LIMIT_MOM);
  DISTIL_CHECK_ARG(v && U && mom && phi && workspace, "distil_meson_elementals: null pointer");
  DISTIL_CHECK_ARG(aligned(v, 8) && aligned(U, 8) && aligned(phi, 16) && aligned(workspace, 256),
                   "distil_meson_elementals: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  const size_t need = meson_elementals_workspace(L, nt, nv, np);
  if (ws_bytes < need) {
    set_error("distil_meson_elementals: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  return meson_elementals(ctx, v, U, L, nt, nv, mom, np, phi, workspace, ws_bytes,
                          reinterpret_cast<cudaStream_t>(stream));
}

int distil_meson_correlate_workspace(int nv, int np, int nb, int mode, size_t* bytes) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(bytes != nullptr, "bytes is null");
  if (mode != DISTIL_MIXED_FP16X6) {
    set_error("distil_meson_correlate_workspace: mode %d not supported (FP16X6 only)", mode);
    return DISTIL_ENOTSUP;
  }
  DISTIL_CHECK_ARG(nv >= 1 && nv <= MS_LIMIT_NV && np >= 1 && np <= MS_LIMIT_MOM && nb >= 1 && nb <= MS_LIMIT_NB,
                   "distil_meson_correlate_workspace: bad sizes");
  *bytes = meson_correlate_workspace(nv, np, nb);
  return DISTIL_OK;
}

int distil_meson_correlate(distil_ctx* ctx, const void* phi_snk, const void* phi_src, const void* tau, int nt,
                           int nv, int np, const double* prof, int nb, int mode, void* C, void* workspace,
                           size_t ws_bytes, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  if (mode != DISTIL_MIXED_FP16X6) {
    set_error("distil_meson_correlate: mode %d not supported (FP16X6 only)", mode);
    return DISTIL_ENOTSUP;
  }
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && nv <= MS_LIMIT_NV, "distil_meson_correlate: nt >= 1, 1 <= nv <= %d",
                   MS_LIMIT_NV);
  DISTIL_CHECK_ARG(np >= 1 && np <= MS_LIMIT_MOM, "distil_meson_correlate: 1 <= np <= %d", MS_LIMIT_MOM);
  DISTIL_CHECK_ARG(nb >= 1 && nb <= MS_LIMIT_NB, "distil_meson_correlate: nb=%d outside [1,%d]", nb, MS_LIMIT_NB);
  DISTIL_CHECK_ARG(phi_snk && phi_src && tau && prof && C && workspace, "distil_meson_correlate: null pointer");
  DISTIL_CHECK_ARG(aligned(phi_snk, 16) && aligned(phi_src, 16) && aligned(tau, 8) && aligned(prof, 8) &&
                       aligned(C, 16) && aligned(workspace, 256),
                   "distil_meson_correlate: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  const size_t need = meson_correlate_workspace(nv, np, nb);
  if (ws_bytes < need) {
    set_error("distil_meson_correlate: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  return meson_correlate(ctx, phi_snk, phi_src, tau, nt, nv, np, prof, nb, C, workspace, ws_bytes,
                         reinterpret_cast<cudaStream_t>(stream));
}

int distil_meson_prune(distil_ctx* ctx, const void* C, int np, int nops, int nt, int t_prune, int nkeep, void* Ct,
                       void* Un, double* sv, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(C && Ct && Un, "distil_meson_prune: null pointer");
  DISTIL_CHECK_ARG(np >= 1 && nt >= 1 && nops >= 1 && nops <= 32, "distil_meson_prune: np, nt >= 1, 1 <= nops <= 32");
  DISTIL_CHECK_ARG(nkeep >= 1 && nkeep <= nops && nkeep <= 16, "distil_meson_prune: 1 <= nkeep <= min(nops, 16)");
  DISTIL_CHECK_ARG(t_prune >= 0 && t_prune < nt, "distil_meson_prune: t_prune=%d outside [0,%d)", t_prune, nt);
  DISTIL_CHECK_ARG(aligned(C, 16) && aligned(Ct, 16) && aligned(Un, 16) && aligned(sv, 8),
                   "distil_meson_prune: misaligned pointer");
  return meson_prune(ctx, C, np, nops, nt, t_prune, nkeep, Ct, Un, sv, reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------- glueball path

int distil_glueball_workspace(int L, int nt, size_t* bytes) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(bytes != nullptr, "bytes is null");
  DISTIL_CHECK_ARG(L >= 2 && L <= MS_LIMIT_L && nt >= 1, "distil_glueball_workspace: 2 <= L <= %d, nt >= 1",
                   MS_LIMIT_L);
  *bytes = glueball_workspace(L, nt);
  return DISTIL_OK;
}

int distil_glueball_operators(distil_ctx* ctx, const void* U, int L, int nt, void* O, void* workspace,
                              size_t ws_bytes, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(L >= 2 && L <= MS_LIMIT_L && nt >= 1, "distil_glueball_operators: 2 <= L <= %d, nt >= 1",
                   MS_LIMIT_L);
  DISTIL_CHECK_ARG(U && O && workspace, "distil_glueball_operators: null pointer");
  DISTIL_CHECK_ARG(aligned(U, 8) && aligned(O, 16) && aligned(workspace, 256),
                   "distil_glueball_operators: misaligned pointer (arrays to their element, workspace to 256 bytes)");
  const size_t need = glueball_workspace(L, nt);
  if (ws_bytes < need) {
    set_error("distil_glueball_operators: workspace %zu < %zu bytes", ws_bytes, need);
    return DISTIL_ENOMEM;
  }
  return glueball_operators(ctx, U, L, nt, O, workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

int distil_mode_supported(int mode) {
  if (!valid_mode(mode)) return 0;
  return is_mixed(mode) ? mixed_mode_built(mode) : 1;
}

int distil_set_tuning(distil_ctx* ctx, const int* variants) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(ctx != nullptr && variants != nullptr, "distil_set_tuning: null pointer");
  for (int i = 0; i < 3; ++i)
    DISTIL_CHECK_ARG(variants[i] >= 0 && variants[i] <= 5 && (i == 0 || variants[i] != 2),
                     "distil_set_tuning: variant %d of site %d", variants[i], i);
  for (int i = 0; i < 3; ++i) ctx->tune[i] = variants[i];
  return DISTIL_OK;
}

int distil_get_tuning(const distil_ctx* ctx, int* variants) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(ctx != nullptr && variants != nullptr, "distil_get_tuning: null pointer");
  for (int i = 0; i < 3; ++i) variants[i] = ctx->tune[i];
  return DISTIL_OK;
}

int distil_device_status(distil_ctx* ctx, int reset, unsigned* code) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CUDA(cudaDeviceSynchronize());
  unsigned w = 0;
  DISTIL_CUDA(cudaMemcpy(&w, ctx->d_error, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (code) *code = w;
  if (reset) DISTIL_CUDA(cudaMemset(ctx->d_error, 0, sizeof(unsigned)));
  if (w) {
    static const char* what[] = {"", "MMA waiting for a copied stage", "copy producer waiting for a free stage",
                                 "epilogue waiting for the accumulator", "teardown waiting for copies in flight"};
    set_error("a bounded device wait expired: %s (code %u)", w < 5 ? what[w] : "unknown", w);
    return DISTIL_ETIMEOUT;
  }
  return DISTIL_OK;
}

int distil_profiles_eigen(distil_ctx* ctx, const double* lam, int nt, int nv, const double* sigma, int nb,
                          double* prof, distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(lam && sigma && prof, "distil_profiles_eigen: null pointer");
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && nb >= 1 && nb <= 16, "distil_profiles_eigen: bad sizes");
  DISTIL_CHECK_ARG(aligned(lam, 8) && aligned(prof, 8), "distil_profiles_eigen: misaligned pointer");
  for (int b = 0; b < nb; ++b)
    DISTIL_CHECK_ARG(sigma[b] > 0.0 && sigma[b] < 1e300, "distil_profiles_eigen: sigma[%d] must be positive", b);
  return eigen_profiles_launch(ctx, lam, nt, nv, sigma, nb, prof, reinterpret_cast<cudaStream_t>(stream));
}

int distil_set_wait_limit(distil_ctx* ctx, long long cycles) {
  g_err[0] = 0;
  DISTIL_CHECK_ARG(ctx != nullptr, "distil_set_wait_limit: null context");
  ctx->wait_limit = cycles > 0 ? cycles : 0;
  return DISTIL_OK;
}

int distil_scan_finite(distil_ctx* ctx, const void* x, long long count, int is_f32, long long* first_bad,
                       distil_stream stream) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(count >= 0 && (x != nullptr || count == 0), "distil_scan_finite: null array");
  DISTIL_CHECK_ARG(aligned(x, is_f32 ? 4 : 8), "distil_scan_finite: misaligned array");
  long long bad = -1;
  DISTIL_TRY(scan_finite_launch(ctx, x, count, is_f32 != 0, &bad, reinterpret_cast<cudaStream_t>(stream)));
  if (first_bad) *first_bad = bad;
  if (bad >= 0) {
    set_error("distil_scan_finite: non-finite value (NaN or Inf) at element %lld", bad);
    return DISTIL_EINVAL;
  }
  return DISTIL_OK;
}

int distil_profile_enable(distil_ctx* ctx, int timing) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  Profiler& p = *ctx->prof;
  DISTIL_CUDA(cudaDeviceSynchronize());
  p.reset();
  p.timing = timing != 0;
  return DISTIL_OK;
}

int distil_profile_read(distil_ctx* ctx, distil_kernel_stat* out, int max, int* count) {
  g_err[0] = 0;
  DISTIL_TRY(enter(ctx));
  DISTIL_CHECK_ARG(count != nullptr && (out != nullptr || max == 0), "distil_profile_read: null pointer");
  Profiler& p = *ctx->prof;
  std::vector<double> ms(p.names.size(), 0.0);
  for (auto& r : p.recs) {
    DISTIL_CUDA(cudaEventSynchronize(r.b));
    float f = 0.f;
    DISTIL_CUDA(cudaEventElapsedTime(&f, r.a, r.b));
    ms[r.kernel] += f;
  }
  int n = (int)p.names.size();
  *count = n;
  for (int i = 0; i < n && i < max; ++i) {
    memset(out[i].name, 0, sizeof(out[i].name));
    strncpy(out[i].name, p.names[i].c_str(), sizeof(out[i].name) - 1);
    out[i].launches = p.launches[i];
    out[i].ms = ms[i];
  }
  return DISTIL_OK;
}

}  // extern "C"
