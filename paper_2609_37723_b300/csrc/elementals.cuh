// Kernel parameters shared by the elemental kernels: momenta and the exact
// phase table exp(-2 pi i m / L), m = 0..L-1 (the phase of site x for
// momentum n is the table entry at (n.x) mod L, so no angle is ever
// formed from a rounded p.x).
#pragma once
#include <math.h>
#include "common.cuh"

namespace distil {

constexpr int EL_MAX_MOM = 64;
constexpr int EL_MAX_L = 256;

template <typename T>
struct ElemParams {
  int L;
  int mom[EL_MAX_MOM][3];
  Cx<T> ptab[EL_MAX_L];
};

template <typename T>
inline void fill_elem_params(ElemParams<T>& prm, int L, const int32_t* mom, int np) {
  prm.L = L;
  for (int q = 0; q < np && q < EL_MAX_MOM; ++q)
    for (int d = 0; d < 3; ++d) prm.mom[q][d] = ((mom[3 * q + d] % L) + L) % L;
  for (int m = 0; m < L && m < EL_MAX_L; ++m) {
    double ang = -2.0 * M_PI * (double)m / (double)L;
    prm.ptab[m] = cmake<T>((T)cos(ang), (T)sin(ang));
  }
}

template <typename T>
int elementals_simt(distil_ctx* ctx, const Cx<T>* v, int L, int nt, int nv, const int32_t* mom, int np, Cx<T>* phi,
                    cudaStream_t stream);

}  // namespace distil
