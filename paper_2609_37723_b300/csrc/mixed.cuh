// Mixed-precision (split 16-bit pieces on tcgen05 tensor cores) paths.
#pragma once
#include "common.cuh"

namespace distil {

int mixed_mode_built(int mode);
size_t elementals_mixed_workspace(int L, int nt, int nv, int np, int mode);
int elementals_mixed(distil_ctx* ctx, const Cx<float>* v, int L, int nt, int nv, const int32_t* mom, int np,
                     int mode, void* phi, void* ws, size_t ws_bytes, cudaStream_t s);

size_t correlate_mixed_workspace(int mode, int nt, int nv, int np, int nb);
int correlate_mixed(distil_ctx* ctx, int mode, const void* phi_snk, const void* phi_src, const void* tau, int nt,
                    int nv, int np, const double* prof_snk, const double* prof_src, int prof_per_t, int nb, void* C,
                    int c_nt, int c_t0, void* ws, size_t ws_bytes, cudaStream_t s);

size_t cgemm_workspace(int mode, long long M, long long N, long long K, long long batch);
int cgemm_mixed(distil_ctx* ctx, int mode, const void* A, const void* B, void* C, int M, int N, int K, int batch,
                void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace distil
