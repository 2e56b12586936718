"""FP64 CPU oracle for the I = 2 two-meson operator built from optimal
one-meson operators.

TEST INFRASTRUCTURE.  Only the tests may import or run this module.  It
shares no code with the CUDA library.

What it computes (paper Sec. 2.3: the optimal one-meson operators of each
GEVP are combined into an I = 2, A1++ two-meson operator with zero total
momentum and back-to-back momenta; no GEVP is solved with it):

* the optimal one-meson operator at momentum p, O_opt(p) = sum_a w_a O_a(p),
  with weights w = U_n u from the pruned GEVP at that momentum (u the GEVP
  eigenvector of the state, U_n the kept singular vectors; oracle.meson);
  its sink matrix M(p, t) = sum_a w_a Phi_a(p, t) and the matrix of its
  adjoint at the source, N(p) = sum_a conj(w_a) Phibar_a(p, 0) =
  gamma_4 M(p, 0)^dagger gamma_4 (spin (x) mode, spin-major);
* the two-meson operator O_2m(t) = sum_{p in P} O_opt(p, t) O_opt(-p, t) over
  the six unit momenta P = {+-e_x, +-e_y, +-e_z} (the A1 sum over the
  directions of a back-to-back pair), both mesons u-bar Gamma d (I = 2);
* its correlator C(t) = <O_2m(t) O_2m(0)^dagger>, by Wick's theorem with the
  forward propagator S = tau(t, 0) and the backward one S~ = g5 S^dagger g5:
      C(t) = sum_{p, p'} [ T(M1, N1) T(M2, N2) + T(M1, N2) T(M2, N1)
                           - X(M1, N1, M2, N2) - X(M1, N2, M2, N1) ]
  with M1 = M(p, t), M2 = M(-p, t), N1 = N(p'), N2 = N(-p'),
  T(M, N) = Tr[M S N S~] and X(A, B, C, D) = Tr[A S B S~ C S D S~] (two
  quark loops: + ; one loop, quark exchange: -).  The one-meson correlator
  of oracle.meson is -T(M, N) in this notation.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import meson

UNIT_MOMENTA = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.int32)


def optimal_weights(C: np.ndarray, t_prune: int, nkeep: int, t0: int, td: int, state: int = 0) -> np.ndarray:
    """Weights w[p][a] of the optimal operator of `state` for every momentum
    of C[p][a][b][t]: w = U_n u, u the right eigenvector of the pruned pencil
    C~(td) u = lambda C~(t0) u with the state-th largest |lambda|, scaled to
    unit norm with its largest component real and positive."""
    Ct, Un, _ = meson.prune(C, t_prune, nkeep)
    out = np.empty((C.shape[0], C.shape[1]), dtype=np.complex128)
    for p in range(C.shape[0]):
        lam, vecs = scipy.linalg.eig(Ct[p, :, :, td], Ct[p, :, :, t0])
        order = np.argsort(-np.abs(lam), kind="stable")
        u = vecs[:, order[state]]
        w = Un[p] @ u
        w = w / np.linalg.norm(w)
        k = int(np.argmax(np.abs(w)))
        out[p] = w * (np.conj(w[k]) / abs(w[k]))
    return out


def sink_operator(phi_q: np.ndarray, prof: np.ndarray, w: np.ndarray) -> np.ndarray:
    """M = sum_a w_a Phi_a for the 3 nb operators a = nb type + sigma."""
    nb = prof.shape[0]
    out = 0
    for typ in range(meson.N_TYPES):
        for s in range(nb):
            out = out + w[typ * nb + s] * meson.sink_matrix(phi_q, prof[s], typ)
    return out


def source_operator(phi0_q: np.ndarray, prof: np.ndarray, w: np.ndarray) -> np.ndarray:
    """N = sum_a conj(w_a) Phibar_a: the matrix of O_opt^dagger at the source."""
    nb = prof.shape[0]
    out = 0
    for typ in range(meson.N_TYPES):
        for s in range(nb):
            out = out + np.conj(w[typ * nb + s]) * meson.source_matrix(phi0_q, prof[s], typ)
    return out


def correlator_t(M: dict, N: dict, tau_t: np.ndarray) -> complex:
    """C(t) of the two-meson operator from the sink matrices M[p] (key: the
    momentum tuple) at t, the source matrices N[p] and tau(t, 0)."""
    tau = np.asarray(tau_t, dtype=np.complex128)
    nv = tau.shape[0] // 4
    G5 = np.kron(meson.GAMMA_5, np.eye(nv))
    back = G5 @ tau.conj().T @ G5
    keys = [tuple(int(x) for x in p) for p in UNIT_MOMENTA]
    neg = lambda p: tuple(-x for x in p)
    # R[p][p'] = M(p) S N(p') S~ for every pair
    R = {(p, q): M[p] @ tau @ N[q] @ back for p in keys for q in keys}
    tr = {k: np.trace(v) for k, v in R.items()}
    C = 0j
    for p in keys:
        for q in keys:
            a, b = (p, q), (neg(p), neg(q))       # M1 N1, M2 N2
            c, d = (p, neg(q)), (neg(p), q)       # M1 N2, M2 N1
            C += tr[a] * tr[b] + tr[c] * tr[d]
            C -= np.sum(R[a] * R[b].T) + np.sum(R[c] * R[d].T)   # Tr[R_a R_b], Tr[R_c R_d]
    return C
