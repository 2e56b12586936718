"""FP64 CPU oracle for the one-meson operators with distillation profiles.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.  It shares no
code, table or layout helper with the CUDA library: it is a plain, slow,
obviously correct restatement of the definitions, in complex128 throughout.

What it computes (paper Sec. 2.3, "Improved charmonium operators": one-meson
operators qbar Gamma q with Gamma in {gamma_0 gamma_5, gamma_0 gamma_5
gamma_i nabla_i, gamma_i BB_i}, each with N_B = 7 Gaussian distillation
profiles, the 21 x 21 correlation matrix pruned to 8 x 8 by the singular
vectors of the 8 largest singular values at a fixed time separation, then a
GEVP):

* the spatial gauge-covariant derivative in direction k, read as the
  symmetric covariant difference
      (nabla_k f)(x) = 1/2 [U_k(x) f(x + k) - U_k(x - k)^dagger f(x - k)]
  on periodic spatial boundaries, and BB_i = eps_ijk nabla_j nabla_k, i.e.
  BB_i = nabla_j nabla_k - nabla_k nabla_j for (i, j, k) cyclic (the
  rightmost derivative acts first);
* the meson elementals with displacement D_d, d = 0..6 standing for
  1, nabla_x, nabla_y, nabla_z, BB_x, BB_y, BB_z:
      Phi^d[p]_ij = sum_x exp(-i p.x) v_i(x)^dagger (D_d v_j)(x)
  (colour inner product; no 1/V3);
* the operator matrices in spin (x) mode space, spin-major like the
  perambulators (index alpha N_v + i), for operator a = 7 type + sigma:
      type 0: gamma_4 gamma_5 (x) g Phi^0 g
      type 1: sum_k gamma_4 gamma_5 gamma_k (x) g Phi^(1+k) g
      type 2: sum_k gamma_k (x) g Phi^(4+k) g
  with g = diag of profile sigma (the profile multiplies both quark
  indices, as the smearing kernel sum_i g_i v_i v_i^dagger does for each
  quark field);  the source (creation) operator is the adjoint
  O^dagger = qbar gamma_4 Gamma^dagger gamma_4 D^dagger q, whose mode
  matrix is (g Phi g)^dagger of the source-time elementals;
* the isovector (connected) correlation matrix with the source at t0 = 0,
      C_ab(p, t) = - Tr[ Phi_a(p, t) tau(t) Phibar_b(p, 0) gamma_5 tau(t)^dagger gamma_5 ],
  the backward propagator from gamma_5-hermiticity; Euclidean gammas in
  the Dirac-Pauli basis, gamma_4 = diag(1, 1, -1, -1), gamma_k with
  off-diagonal blocks -+ i sigma_k, gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4;
* pruning: C(t_p) = U S V^dagger (SVD), U_n = the columns of the n largest
  singular values, Ct(t) = U_n^dagger C(t) U_n for every t (the left
  singular vectors on both sides, so a Hermitian C stays Hermitian);
* the GEVP of the pruned pencil, by the nucleon oracle's gevp.

Layouts shared with the library's C interface (inputs and outputs only):
v[t][i][s][a], s = x + L(y + Lz); U[t][k][s][a][b]; tau[t][alpha N_v + i]
[alpha' N_v + i']; profiles prof[sigma][i]; elementals phi[t][p][d][i][j];
C[p][a][b][t].
"""
from __future__ import annotations

import numpy as np

from . import nucleon

N_DISP = 7
N_TYPES = 3

# ---------------------------------------------------------------------------
# Gamma matrices (Euclidean, Dirac-Pauli basis)
# ---------------------------------------------------------------------------

_SIGMA = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
          np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          np.array([[1, 0], [0, -1]], dtype=np.complex128)]
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)

GAMMA_K = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _SIGMA]
GAMMA_4 = np.block([[_I2, _Z2], [_Z2, -_I2]])
GAMMA_5 = GAMMA_K[0] @ GAMMA_K[1] @ GAMMA_K[2] @ GAMMA_4


def operator_terms(typ: int):
    """[(displacement d, Gamma)] of operator type 0, 1 or 2."""
    g45 = GAMMA_4 @ GAMMA_5
    if typ == 0:
        return [(0, g45)]
    if typ == 1:
        return [(1 + k, g45 @ GAMMA_K[k]) for k in range(3)]
    if typ == 2:
        return [(4 + k, GAMMA_K[k]) for k in range(3)]
    raise ValueError(typ)


# ---------------------------------------------------------------------------
# Covariant derivatives
# ---------------------------------------------------------------------------


def _shift_field(f: np.ndarray, L: int, k: int, step: int) -> np.ndarray:
    """g(x) = f(x + step e_k) for a field f[n][V3][3] on the periodic L^3
    lattice, s = x + L(y + Lz): the site axis seen as (z, y, x)."""
    n = f.shape[0]
    g = f.reshape(n, L, L, L, 3)
    return np.roll(g, -step, axis=3 - k).reshape(f.shape)


def _shift_link(u: np.ndarray, L: int, k: int, step: int) -> np.ndarray:
    """g(x) = u(x + step e_k) for one direction's links u[V3][3][3]."""
    g = u.reshape(L, L, L, 3, 3)
    return np.roll(g, -step, axis=2 - k).reshape(u.shape)


def nabla(U_t: np.ndarray, f: np.ndarray, L: int, k: int) -> np.ndarray:
    """(nabla_k f)(x) = 1/2 [U_k(x) f(x+k) - U_k(x-k)^dagger f(x-k)] for
    fields f[n][V3][3] and links U_t[3][V3][3][3] of one timeslice."""
    Uk = np.asarray(U_t[k], dtype=np.complex128)
    f = np.asarray(f, dtype=np.complex128)
    fwd = np.einsum("sab,nsb->nsa", Uk, _shift_field(f, L, k, +1))
    Ub = _shift_link(Uk, L, k, -1)  # U_k(x - k)
    bwd = np.einsum("sba,nsb->nsa", Ub.conj(), _shift_field(f, L, k, -1))
    return 0.5 * (fwd - bwd)


def bb(U_t: np.ndarray, f: np.ndarray, L: int, i: int) -> np.ndarray:
    """BB_i f = eps_ijk nabla_j nabla_k f = nabla_j (nabla_k f) - nabla_k (nabla_j f)."""
    j, k = (i + 1) % 3, (i + 2) % 3
    return nabla(U_t, nabla(U_t, f, L, k), L, j) - nabla(U_t, nabla(U_t, f, L, j), L, k)


def displaced(U_t: np.ndarray, v_t: np.ndarray, L: int) -> np.ndarray:
    """D_d v_j for d = 0..6 (1, nabla_x,y,z, BB_x,y,z): [7][n][V3][3]."""
    v = np.asarray(v_t, dtype=np.complex128)
    out = [v]
    out += [nabla(U_t, v, L, k) for k in range(3)]
    out += [bb(U_t, v, L, i) for i in range(3)]
    return np.stack(out)


# ---------------------------------------------------------------------------
# Elementals
# ---------------------------------------------------------------------------


def elementals_t(v_t: np.ndarray, U_t: np.ndarray, L: int, mom: np.ndarray) -> np.ndarray:
    """Phi^d[p]_ij = sum_x exp(-i p.x) v_i(x)^dagger (D_d v_j)(x): [np][7][nv][nv]."""
    v = np.asarray(v_t, dtype=np.complex128)
    nv = v.shape[0]
    W = displaced(U_t, v, L).reshape(N_DISP * nv, -1)  # rows (d, j), columns (s, a)
    ph = nucleon.momentum_phases(L, mom)              # [np][V3], exp(-i p.x)
    out = np.empty((len(ph), N_DISP, nv, nv), dtype=np.complex128)
    for q in range(len(ph)):
        A = (ph[q][None, :, None] * v.conj()).reshape(nv, -1)  # rows i
        out[q] = (A @ W.T).reshape(nv, N_DISP, nv).transpose(1, 0, 2)
    return out


def elementals(v: np.ndarray, U: np.ndarray, L: int, mom: np.ndarray) -> np.ndarray:
    """phi[t][p][d][i][j] for every timeslice."""
    return np.stack([elementals_t(v[t], U[t], L, mom) for t in range(v.shape[0])])


# ---------------------------------------------------------------------------
# Correlation matrix
# ---------------------------------------------------------------------------


def sink_matrix(phi_q: np.ndarray, g: np.ndarray, typ: int) -> np.ndarray:
    """Phi_a = sum_c Gamma_c (x) g Phi^(d_c) g, [4nv][4nv] spin-major."""
    out = 0
    for d, G in operator_terms(typ):
        out = out + np.kron(G, g[:, None] * phi_q[d] * g[None, :])
    return out


def source_matrix(phi0_q: np.ndarray, g: np.ndarray, typ: int) -> np.ndarray:
    """Phibar_b = sum_c gamma_4 Gamma_c^dagger gamma_4 (x) (g Phi^(d_c)(0) g)^dagger."""
    out = 0
    for d, G in operator_terms(typ):
        Gbar = GAMMA_4 @ G.conj().T @ GAMMA_4
        out = out + np.kron(Gbar, (g[:, None] * phi0_q[d] * g[None, :]).conj().T)
    return out


def correlator_t(phi_t: np.ndarray, phi_src: np.ndarray, tau_t: np.ndarray, prof: np.ndarray) -> np.ndarray:
    """C[p][a][b] at one sink timeslice: -Tr[Phi_a tau Phibar_b g5 tau^dagger g5]."""
    npm, _, nv, _ = phi_t.shape
    nb = prof.shape[0]
    tau = np.asarray(tau_t, dtype=np.complex128)
    G5 = np.kron(GAMMA_5, np.eye(nv))
    back = G5 @ tau.conj().T @ G5  # tau(0, t) from gamma_5-hermiticity
    nops = N_TYPES * nb
    C = np.empty((npm, nops, nops), dtype=np.complex128)
    for q in range(npm):
        P = np.stack([sink_matrix(phi_t[q], prof[s], typ) @ tau
                      for typ in range(N_TYPES) for s in range(nb)])
        R = np.stack([source_matrix(phi_src[q], prof[s], typ) @ back
                      for typ in range(N_TYPES) for s in range(nb)])
        # Tr[P_a R_b] = sum_ij P_a[i][j] R_b[j][i]
        C[q] = -(P.reshape(nops, -1) @ R.transpose(0, 2, 1).reshape(nops, -1).T)
    return C


def correlator(phi: np.ndarray, phi_src: np.ndarray, tau: np.ndarray, prof: np.ndarray) -> np.ndarray:
    """C[p][a][b][t] for the sink timeslices of phi[t] and tau[t]."""
    return np.stack([correlator_t(phi[t], phi_src, tau[t], prof) for t in range(phi.shape[0])], axis=-1)


# ---------------------------------------------------------------------------
# Pruning and GEVP
# ---------------------------------------------------------------------------


def prune(C: np.ndarray, t_prune: int, n: int):
    """Ct[p][:n][:n][t] = U_n^dagger C(t) U_n with U_n the left singular
    vectors of C(t_prune) of the n largest singular values.  Returns
    (Ct, U_n [p][nops][n], singular values [p][nops], descending)."""
    npm, nops, _, nt = C.shape
    Ct = np.empty((npm, n, n, nt), dtype=np.complex128)
    Un = np.empty((npm, nops, n), dtype=np.complex128)
    sv = np.empty((npm, nops))
    for p in range(npm):
        u, s, _ = np.linalg.svd(C[p, :, :, t_prune])
        Un[p] = u[:, :n]
        sv[p] = s
        for t in range(nt):
            Ct[p, :, :, t] = Un[p].conj().T @ C[p, :, :, t] @ Un[p]
    return Ct, Un, sv


def gevp(C: np.ndarray, t0: int) -> np.ndarray:
    """Generalized eigenvalues of the (pruned) pencil, sorted by |lambda|."""
    return nucleon.gevp(C, t0)
