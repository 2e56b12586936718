// TMA tensor-map encoding for the tensor-core GEMM (driver entry point
// cuTensorMapEncodeTiled, looked up once through the runtime).
#include <cuda.h>

#include "tc_host.cuh"

namespace distil {
namespace tc {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int encode_planes(CUtensorMap* map, const Planes& t, int box_rows, int kc, bool bf16) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return DISTIL_ECUDA;
  }
  if ((reinterpret_cast<uintptr_t>(t.base) & 15) || (t.ld * 2) % 16 || (t.plane_stride * 2) % 16 ||
      (t.batch_stride * 2) % 16) {
    set_error("encode_planes: base/strides not 16-byte aligned");
    return DISTIL_EINVAL;
  }
  cuuint64_t dims[4] = {(cuuint64_t)t.K, (cuuint64_t)t.rows, (cuuint64_t)t.planes, (cuuint64_t)t.batch};
  cuuint64_t strides[3] = {(cuuint64_t)(t.ld * 2), (cuuint64_t)(t.plane_stride * 2),
                           (cuuint64_t)(t.batch_stride * 2)};
  cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)box_rows, (cuuint32_t)t.planes, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUtensorMapSwizzle swz = kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                           : kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                      : CU_TENSOR_MAP_SWIZZLE_32B;
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, t.base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): K=%lld rows=%lld planes=%lld batch=%lld box_rows=%d kc=%d",
              (int)r, t.K, t.rows, t.planes, t.batch, box_rows, kc);
    return DISTIL_ECUDA;
  }
  return DISTIL_OK;
}

}  // namespace tc
}  // namespace distil
