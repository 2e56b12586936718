// Placeholder for the tensor-core paths until they are built.
#include "mixed.cuh"

namespace distil {

int mixed_mode_built(int) { return 0; }
size_t elementals_mixed_workspace(int, int, int, int, int) { return 0; }
int elementals_mixed(distil_ctx*, const Cx<float>*, int, int, int, const int32_t*, int, int, Cx<float>*, void*,
                     size_t, cudaStream_t) {
  set_error("mixed-precision elementals not built");
  return DISTIL_ENOTSUP;
}
size_t correlate_mixed_workspace(int, int, int) { return 0; }
int correlate_mixed(distil_ctx*, int, const void*, const void*, const void*, int, int, int, const double*, int, int,
                    void*, void*, size_t, cudaStream_t) {
  set_error("mixed-precision correlator not built");
  return DISTIL_ENOTSUP;
}

}  // namespace distil
