// The correlation matrix as three mode contractions (shared by all modes).
//
// With Gamma = C gamma_5, P+ = diag(1,1,0,0) and Psi^(a)mu as in distil.h,
// the definition of C_ab(t) regroups exactly into
//
//   U^a_{(a'i')(beta j) k} = Gamma_{alpha(beta) beta} sum_i tau_{(alpha(beta) i)(a'i')} G^a_{ijk}
//   V^a_{(a'i')(b'j') k}   = sum_{beta j} tau_{(beta j)(b'j')} U^a_{(a'i')(beta j) k}
//   X^{b,c}_{i'j' k}       = sum_k' T^c_{k k'} conj(G^b_{i'j'k'})
//   C_ab = sum_terms coef * sum_{i'<j',k} (V^a_{i'j'k} - V^a_{j'i'k}) X^{b,c}_{i'j'k}
//
// where G^a = g^a g^a g^a Phi, alpha(beta) = beta xor 1 is the only row with
// Gamma_{alpha beta} != 0, and the 14 source spin triples of the direct
// minus exchange bracket collapse onto six sink-side spin pairs (a',b') and
// five source matrices T^c: the triples with a' = b' drop out (V symmetric,
// X antisymmetric in i'j'), a triple with a' > b' maps onto (b', a') with a
// sign, and T^+ = tau^{00} + tau^{11} merges the two projector rows.  The
// sink-side contractions (i, then j) are shared by every source profile b,
// the source side (k') by every sink profile a; the final dot is the only
// N_B^2 piece.
#pragma once
#include "common.cuh"

namespace distil {

// Spin pairs (a', b') kept on the sink side, in storage order.
constexpr int NPAIR = 6;
__host__ __device__ constexpr int pair_ap(int s) { return s < 3 ? 0 : (s < 5 ? 1 : 2); }
__host__ __device__ constexpr int pair_bp(int s) { return s < 3 ? s + 1 : (s < 5 ? s - 1 : 3); }
// Source matrices: 0 = tau^{00}+tau^{11}, 1 = tau^{02}, 2 = tau^{03}, 3 = tau^{12}, 4 = tau^{13}.
constexpr int NSRC = 5;
// The six surviving terms: (pair slot, source matrix, coefficient).
//   (0,1) with T^+ : -3  [(0,1,mu): -2 direct+exchange (mu=0) / -1 (mu=1);
//                        mirror (1,0,mu): -1 (mu=0) / -2 (mu=1)]
//   (2,3) with T^+ : -2  [(2,3,mu): -1; mirror (3,2,mu): -1]
//   (0,3) with tau^{02}: -1,  (0,2) with tau^{03}: +1,
//   (1,3) with tau^{12}: -1,  (1,2) with tau^{13}: +1.
constexpr int NTERM = 6;
__host__ __device__ constexpr int dot_slot(int t) {
  return t == 0 ? 0 : t == 1 ? 5 : t == 2 ? 2 : t == 3 ? 1 : t == 4 ? 4 : 3;
}
__host__ __device__ constexpr int dot_src(int t) { return t == 0 || t == 1 ? 0 : t - 1; }
__host__ __device__ constexpr double dot_coef(int t) {
  return t == 0 ? -3.0 : t == 1 ? -2.0 : (t == 2 || t == 4) ? -1.0 : 1.0;
}

// Both paths compute C for the call's nt sink timeslices t into
// C[q][a][b][c_t0 + t] of an array with c_nt timeslices (other columns are
// not touched).  Sink timeslice t uses the profiles prof_snk (+ t nb nv when
// prof_per_t), the source prof_src.
int correlate_plain(distil_ctx* ctx, int fp64, const void* phi_snk, const void* phi_src, const void* tau,
                    int nt, int nv, int np, const double* prof_snk, const double* prof_src, int prof_per_t, int nb,
                    void* C, int c_nt, int c_t0, void* ws, size_t ws_bytes, cudaStream_t s);

// Zero the columns [c_t0, c_t0 + nt) of `rows` rows of c_nt complex128 values.
inline int zero_c_columns(void* C, long long rows, int c_nt, int c_t0, int nt, cudaStream_t s) {
  const size_t e = sizeof(double) * 2;
  DISTIL_CUDA(cudaMemset2DAsync(static_cast<char*>(C) + e * c_t0, e * c_nt, 0, e * nt, (size_t)rows, s));
  return DISTIL_OK;
}
size_t correlate_plain_workspace(int fp64, int nv, int nb);

}  // namespace distil
