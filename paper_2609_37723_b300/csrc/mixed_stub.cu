// Placeholder for the tensor-core elementals until they are built.
#include "mixed.cuh"

namespace distil {

size_t elementals_mixed_workspace(int, int, int, int, int) { return 0; }
int elementals_mixed(distil_ctx*, const Cx<float>*, int, int, int, const int32_t*, int, int, Cx<float>*, void*,
                     size_t, cudaStream_t) {
  set_error("mixed-precision elementals not built");
  return DISTIL_ENOTSUP;
}

}  // namespace distil
