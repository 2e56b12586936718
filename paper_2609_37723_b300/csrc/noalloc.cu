// distil_correlate_noalloc: the plain correlation matrix with its scratch in
// a fixed device array instead of caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need
// the correlation matrix: a process running under a fixed device-memory
// budget that was reserved up front, or a latency-critical pipeline that
// cannot afford the device-wide synchronisation cudaMalloc and cudaFree may
// imply.  This entry point calls no allocating routine at all.  Its scratch
// is the file-scope device array below; every GPU that loads the library
// holds it until the process exits.
#include <mutex>

#include "common.cuh"
#include "correlate.cuh"

namespace distil {

// Largest scratch the entry point accepts: 16 MiB.  FP64 needs about
// 352 N_B N_v^3 bytes (the exact count is correlate_plain_workspace): N_v = 16
// fits with N_B <= 11, N_v = 20 with N_B <= 5, N_v = 24 with N_B <= 3.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in, so the real
// address is looked up with cudaGetSymbolAddress.  The lookup is repeated on
// every call made outside stream capture (it is cheap, and a cudaDeviceReset
// in between reloads the module at a possibly different address); a call
// made while `stream` is being captured uses the address cached by the last
// uncaptured call on that device, and fails if there was none.
static int noalloc_scratch(int device, cudaStream_t stream, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) {
    set_error("distil_correlate_noalloc: device %d out of range", device);
    return DISTIL_EINVAL;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DISTIL_CUDA(cudaStreamIsCapturing(stream, &cap));
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("distil_correlate_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return DISTIL_ECUDA;
    }
    g_noalloc_addr[device] = p;
  } else if (!g_noalloc_addr[device]) {
    set_error("distil_correlate_noalloc: first call on device %d made during stream capture", device);
    return DISTIL_EINVAL;
  }
  *out = g_noalloc_addr[device];
  return DISTIL_OK;
}

static bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace distil

using namespace distil;

extern "C" int distil_correlate_noalloc(distil_ctx* ctx, const void* phi_snk, const void* phi_src, const void* tau,
                                        int nt, int nv, int np, const double* prof, int nb, int prof_per_t,
                                        int mode, void* C, distil_stream stream) {
  set_error("%s", "");
  DISTIL_CHECK_ARG(ctx != nullptr, "distil_correlate_noalloc: null context");
  DISTIL_CHECK_ARG(mode == DISTIL_FP64 || mode == DISTIL_FP32,
                   "distil_correlate_noalloc: mode %d not supported (FP64 or FP32 only)", mode);
  DISTIL_CHECK_ARG(nt >= 1 && nv >= 1 && np >= 1, "distil_correlate_noalloc: nt, nv, np must be >= 1");
  DISTIL_CHECK_ARG(nb >= 1 && nb <= 16, "distil_correlate_noalloc: nb=%d outside [1,16]", nb);
  DISTIL_CHECK_ARG(tau && prof && C && ((phi_snk && phi_src) || comb3(nv) == 0),
                   "distil_correlate_noalloc: null pointer");
  DISTIL_CHECK_ARG(aligned_to(phi_snk, mode == DISTIL_FP32 ? 8 : 16) && aligned_to(phi_src, mode == DISTIL_FP32 ? 8 : 16) &&
                       aligned_to(tau, mode == DISTIL_FP64 ? 16 : 8) && aligned_to(prof, 8) && aligned_to(C, 16),
                   "distil_correlate_noalloc: misaligned pointer (arrays must be aligned to their element, C to 16 bytes)");
  const size_t need = correlate_plain_workspace(mode == DISTIL_FP64, nv, nb);
  if (nv >= 3 && need > NOALLOC_SCRATCH_BYTES) {
    set_error("distil_correlate_noalloc: N_v=%d, N_B=%d need %zu bytes of scratch, more than its %zu-byte array",
              nv, nb, need, NOALLOC_SCRATCH_BYTES);
    return DISTIL_ENOMEM;
  }
  DISTIL_CUDA(cudaSetDevice(ctx->device));
  void* scratch = nullptr;
  DISTIL_TRY(noalloc_scratch(ctx->device, reinterpret_cast<cudaStream_t>(stream), &scratch));
  // no context: no launch bookkeeping, nothing allocated on the host either
  return correlate_plain(nullptr, mode == DISTIL_FP64, phi_snk, phi_src, tau, nt, nv, np, prof, prof, prof_per_t, nb,
                         C, nt, 0, scratch, NOALLOC_SCRATCH_BYTES, reinterpret_cast<cudaStream_t>(stream));
}
