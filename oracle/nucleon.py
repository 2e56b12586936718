"""FP64 CPU oracle for the distilled-nucleon hot path.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.  It shares no
code, table or layout helper with the CUDA library: it is a plain, slow,
obviously correct restatement of the definitions, in complex128 throughout.

What it computes (paper Sec. 2.1, "Improved nucleon operators"):

* the nucleon elementals ("triplets")
      Phi[p,t]_ijk = sum_x exp(-i p.x) eps_abc v_i^a(x,t) v_j^b(x,t) v_k^c(x,t)
  from N_v distillation vectors per timeslice.  The paper names Phi[p,t]_ijk
  but prints no formula for it; this is the standard baryon elemental with no
  displacement and no 1/V3 factor.  The colour sum is the scalar triple
  product det[v_i, v_j, v_k] = v_i . (v_j x v_k), written out term by term.
* the profile rescaling of the paper's displayed equation in Sec. 2.1,
      Phi^(a)_ijk = g_i^(a) g_j^(a) g_k^(a) Phi_ijk   (no sums),
* the N_B x N_B correlation matrix of the profiled elementals, with the
  spin structure the paper omits taken as the positive-parity nucleon
  N_mu = eps (u^T C gamma_5 d) u_mu, projector P+ = (1 + gamma_4)/2 in the
  Dirac-Pauli basis, quark slots u(i) d(j) u(k), source at t0 = 0, and both
  Wick orderings of the two u quarks (direct minus exchange):
      C_ab(t) = sum_{mu nu} P_{nu mu} sum Psi^(a)mu_{IJK}(t) tau_II' tau_JJ' tau_KK'
                [Psi^(b)nu_{I'J'K'}(0) - Psi^(b)nu_{K'J'I'}(0)]^*
  with I = (alpha, i) and Psi^(a)mu_{(alpha i)(beta j)(gamma k)}
  = Phi^(a)_ijk Gamma_{alpha beta} delta_{gamma mu}.  By the antisymmetry of
  Phi the bracket is Phi^(b)* times the spin tensor
  s^nu_{a'b'c'} = Gamma_{a'b'} delta_{c' nu} + Gamma_{c'b'} delta_{a' nu};
  the tests check this folding against the unfolded two-term form.
  The sum over I'J'K' is done as three successive mode contractions, first
  k', then j', then i', as the method prescribes.
* the generalized eigenvalue problem C(t) u = lambda C(t0) u on each N_B x N_B
  matrix (Sec. 2.1: "solve a GEVP"), eigenvalues sorted by |lambda|,
  largest first.

Layouts shared with the library's C interface (inputs and outputs only):
v[t][i][s][a] with s = x + L(y + Lz); packed triples i<j<k at colex rank
C(k,3) + C(j,2) + i; tau[t][alpha*N_v + i][alpha'*N_v + i'];
C[p][a][b][t].
"""
from __future__ import annotations

import math
from typing import Iterable, Optional, Sequence

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------
# Index bookkeeping
# ---------------------------------------------------------------------------


def n_triples(nv: int) -> int:
    return nv * (nv - 1) * (nv - 2) // 6


def triple_rank(i: int, j: int, k: int) -> int:
    """Colex rank of i<j<k: C(k,3) + C(j,2) + i."""
    return math.comb(k, 3) + math.comb(j, 2) + i


def triples(nv: int):
    """(i, j, k) arrays of all i<j<k in rank order."""
    out = [(i, j, k) for k in range(nv) for j in range(k) for i in range(j)]
    a = np.array(out, dtype=np.int64).reshape(-1, 3)
    return a[:, 0], a[:, 1], a[:, 2]


def unpack(phi_packed: np.ndarray, nv: int) -> np.ndarray:
    """Dense antisymmetric [..., nv, nv, nv] tensor from packed i<j<k values."""
    i, j, k = triples(nv)
    lead = phi_packed.shape[:-1]
    d = np.zeros(lead + (nv, nv, nv), dtype=np.complex128)
    f = phi_packed.astype(np.complex128)
    for (a, b, c), sgn in (((i, j, k), 1), ((j, k, i), 1), ((k, i, j), 1),
                           ((j, i, k), -1), ((i, k, j), -1), ((k, j, i), -1)):
        d[..., a, b, c] = sgn * f
    return d


# ---------------------------------------------------------------------------
# Elementals
# ---------------------------------------------------------------------------


def site_coords(L: int) -> np.ndarray:
    s = np.arange(L ** 3)
    return np.stack([s % L, (s // L) % L, s // (L * L)], axis=1)


def momentum_phases(L: int, mom: np.ndarray) -> np.ndarray:
    """exp(-i p.x) with p = 2 pi n / L, as [np][V3]."""
    xyz = site_coords(L)
    m = (np.asarray(mom, dtype=np.int64) @ xyz.T) % L
    return np.exp(-2j * np.pi * m / L)


def elementals_t(v_t: np.ndarray, L: int, mom: np.ndarray) -> np.ndarray:
    """Phi[p]_ijk for one timeslice, packed i<j<k: [np][T3].

    v_t: [nv][V3][3].  For each k the colour cross products
    w_jk = v_j x v_k (j < k) are formed site by site; then
    Phi_ijk(p) = sum_{x,a} exp(-ip.x) v_i^a(x) w_jk^a(x), i.e. the triple
    product eps_abc v_i^a v_j^b v_k^c summed over sites with the phase.
    """
    v = v_t.astype(np.complex128)
    nv, V3, _ = v.shape
    ph = momentum_phases(L, mom)                      # [np][V3]
    npm = ph.shape[0]
    # E[(p,i)][(x,a)] = exp(-ip.x) v_i^a(x)
    E = (ph[:, None, :, None] * v[None, :, :, :]).reshape(npm * nv, V3 * 3)
    out = np.zeros((npm, n_triples(nv)), dtype=np.complex128)
    for k in range(2, nv):
        vj = v[:k]                                     # [k][V3][3]
        vk = v[k]                                      # [V3][3]
        w = np.empty_like(vj)
        w[..., 0] = vj[..., 1] * vk[None, :, 2] - vj[..., 2] * vk[None, :, 1]
        w[..., 1] = vj[..., 2] * vk[None, :, 0] - vj[..., 0] * vk[None, :, 2]
        w[..., 2] = vj[..., 0] * vk[None, :, 1] - vj[..., 1] * vk[None, :, 0]
        phi_pij = (E @ w.reshape(k, V3 * 3).T).reshape(npm, nv, k)   # [p][i][j]
        for j in range(1, k):
            r0 = math.comb(k, 3) + math.comb(j, 2)
            out[:, r0:r0 + j] = phi_pij[:, :j, j]
    return out


def elementals(v: np.ndarray, L: int, mom: np.ndarray) -> np.ndarray:
    """Phi[t][p][T3] for all timeslices of v[t][nv][V3][3]."""
    return np.stack([elementals_t(v[t], L, mom) for t in range(v.shape[0])])


# ---------------------------------------------------------------------------
# Spin structure
# ---------------------------------------------------------------------------

# Dirac-Pauli basis, Euclidean gammas: gamma_4 = diag(1,1,-1,-1);
# C = gamma_2 gamma_4; Gamma = C gamma_5 = [[0,-1],[1,0]] (+) [[0,-1],[1,0]].
GAMMA = np.array([[0, -1, 0, 0],
                  [1, 0, 0, 0],
                  [0, 0, 0, -1],
                  [0, 0, 1, 0]], dtype=np.float64)
P_PLUS = np.diag([1.0, 1.0, 0.0, 0.0])


def sink_spin(mu: int) -> dict:
    """Nonzero components of Gamma_{alpha beta} delta_{gamma mu}."""
    out = {}
    for a in range(4):
        for b in range(4):
            if GAMMA[a, b] != 0:
                out[(a, b, mu)] = GAMMA[a, b]
    return out


def source_spin(nu: int) -> dict:
    """s^nu_{a'b'c'} = Gamma_{a'b'} delta_{c' nu} + Gamma_{c'b'} delta_{a' nu}:
    the direct minus exchange source bracket divided by conj(Phi^(b))."""
    s = {}
    for a in range(4):
        for b in range(4):
            for c in range(4):
                val = GAMMA[a, b] * (c == nu) + GAMMA[c, b] * (a == nu)
                if val != 0:
                    s[(a, b, c)] = val
    return s


# ---------------------------------------------------------------------------
# Correlation matrix
# ---------------------------------------------------------------------------


def eigenvalue_profiles(lam: np.ndarray, sigmas) -> np.ndarray:
    """Quark distillation profiles as functions of the Laplacian eigenvalues
    (Sec. 2.1: the profiles "can be a function of the 3D Laplacian
    eigenvalues"), Gaussian in the eigenvalue:
        g^(b)_i[t] = exp(-(lam_i[t] / sigma_b)^2).
    lam: [nv] or [nt][nv]; returns [nb][nv] or [nt][nb][nv]."""
    lam = np.asarray(lam, dtype=np.float64)
    sig = np.asarray(sigmas, dtype=np.float64)
    return np.exp(-(lam[..., None, :] / sig[:, None]) ** 2)


def profile_scale(phi_dense: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Phi^(a)_ijk = g_i g_j g_k Phi_ijk (no sum)."""
    return phi_dense * g[:, None, None] * g[None, :, None] * g[None, None, :]


def correlator_tp(phi_snk: np.ndarray, phi_src: np.ndarray, tau: np.ndarray,
                  g_snk: np.ndarray, g_src: np.ndarray,
                  bs: Optional[Iterable[int]] = None) -> np.ndarray:
    """C_ab at one (t, p): [nb][nb] (columns outside ``bs`` left zero).

    phi_snk: packed [T3] at time t; phi_src: packed [T3] at t0 = 0;
    tau: [4nv][4nv] = tau(t, t0); g_snk, g_src: [nb][nv] profiles at t, t0.
    """
    nv = tau.shape[0] // 4
    nb = g_snk.shape[0]
    tau = tau.astype(np.complex128)
    dense_snk = unpack(phi_snk, nv)
    dense_src = unpack(phi_src, nv)

    def blk(a, b):
        return tau[a * nv:(a + 1) * nv, b * nv:(b + 1) * nv]

    C = np.zeros((nb, nb), dtype=np.complex128)
    bs = range(nb) if bs is None else bs
    for b in bs:
        S = np.conj(profile_scale(dense_src, g_src[b]))          # [i'][j'][k']
        for nu in range(4):
            for mu in range(4):
                if P_PLUS[nu, mu] == 0:
                    continue
                snk = sink_spin(mu)
                R = {key: np.zeros((nv, nv, nv), dtype=np.complex128) for key in snk}
                for (ap, bp, cp), s in source_spin(nu).items():
                    # k' first: X[i',j',k] = sum_k' tau^{mu c'}_{k k'} S[i',j',k']
                    X = (S.reshape(nv * nv, nv) @ blk(mu, cp).T).reshape(nv, nv, nv)
                    for (a, bb, c) in snk:
                        # then j': Y[i',j,k] = sum_j' tau^{bb b'}_{j j'} X[i',j',k]
                        Y = np.matmul(blk(bb, bp), X)
                        # then i': Z[i,j,k] = sum_i' tau^{a a'}_{i i'} Y[i',j,k]
                        Z = (blk(a, ap) @ Y.reshape(nv, nv * nv)).reshape(nv, nv, nv)
                        R[(a, bb, c)] += s * Z
                for a_ in range(nb):
                    G = profile_scale(dense_snk, g_snk[a_])
                    acc = 0j
                    for key, w in snk.items():
                        acc += w * np.sum(G * R[key])
                    C[a_, b] += P_PLUS[nu, mu] * acc
    return C


def correlator(phi_snk: np.ndarray, phi_src: np.ndarray, tau: np.ndarray,
               prof: np.ndarray, prof_per_t: bool = False,
               ts: Optional[Sequence[int]] = None, ps: Optional[Sequence[int]] = None) -> np.ndarray:
    """C[p][a][b][t] for phi_snk [nt][np][T3], phi_src [np][T3], tau [nt][4nv][4nv],
    prof [nb][nv] (or [nt][nb][nv] when prof_per_t).  Entries outside the
    requested (ts, ps) stay zero."""
    nt, npm = phi_snk.shape[0], phi_snk.shape[1]
    nb = prof.shape[-2]
    C = np.zeros((npm, nb, nb, nt), dtype=np.complex128)
    ts = range(nt) if ts is None else ts
    ps = range(npm) if ps is None else ps
    for t in ts:
        g_snk = prof[t] if prof_per_t else prof
        g_src = prof[0] if prof_per_t else prof
        for p in ps:
            C[p, :, :, t] = correlator_tp(phi_snk[t, p], phi_src[p], tau[t], g_snk, g_src)
    return C


# ---------------------------------------------------------------------------
# GEVP
# ---------------------------------------------------------------------------


def gevp(C: np.ndarray, t0: int) -> np.ndarray:
    """Generalized eigenvalues of C(t) u = lambda C(t0) u for every (p, t):
    lambda[p][t][nb], sorted by |lambda| descending."""
    npm, nb, _, nt = C.shape
    lam = np.zeros((npm, nt, nb), dtype=np.complex128)
    for p in range(npm):
        A0 = C[p, :, :, t0]
        for t in range(nt):
            w = scipy.linalg.eigvals(C[p, :, :, t], A0)
            lam[p, t] = w[np.argsort(-np.abs(w), kind="stable")]
    return lam


def _unit_phase(u: np.ndarray) -> np.ndarray:
    """Scale a vector to unit 2-norm and rotate its phase so that its
    largest-modulus component (the first of equal ones) is real positive."""
    u = u / np.linalg.norm(u)
    k = int(np.argmax(np.abs(u)))
    return u * (np.conj(u[k]) / abs(u[k]))


def gevp_vectors(C: np.ndarray, t0: int):
    """Generalized eigenvalues and right eigenvectors of C(t) u = lambda C(t0) u
    for every (p, t) (Sec. 2.1: the GEVP whose eigenvectors give the optimal
    combination of the N_B profiled operators), by scipy.linalg.eig.
    Returns lam[p][t][n] sorted by |lambda| descending and vecs[p][t][n][:],
    each eigenvector of unit norm with its largest component real positive."""
    npm, nb, _, nt = C.shape
    lam = np.zeros((npm, nt, nb), dtype=np.complex128)
    vecs = np.zeros((npm, nt, nb, nb), dtype=np.complex128)
    for p in range(npm):
        for t in range(nt):
            w, u = scipy.linalg.eig(C[p, :, :, t], C[p, :, :, t0])
            order = np.argsort(-np.abs(w), kind="stable")
            lam[p, t] = w[order]
            for n, col in enumerate(order):
                vecs[p, t, n] = _unit_phase(u[:, col])
    return lam, vecs


def optimal_correlator(C: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Correlator of the optimal operators: C_n(t) = u_n^H C(t) u_n for the
    eigenvectors u[p][n][:] of one GEVP (Sec. 2.1: the profiled operators
    combined with the GEVP eigenvector weights).  Returns [p][n][t]."""
    npm, nb, _, nt = C.shape
    out = np.zeros((npm, nb, nt), dtype=np.complex128)
    for p in range(npm):
        for n in range(nb):
            for t in range(nt):
                out[p, n, t] = np.vdot(u[p, n], C[p, :, :, t] @ u[p, n])
    return out


def effective_mass(Cn: np.ndarray) -> np.ndarray:
    """m_eff(t) = log(|C(t)| / |C(t+1)|) along the last axis (lattice units;
    the moduli make it defined for the complex correlators of synthetic
    inputs).  The last timeslice has no partner and gets NaN."""
    a = np.abs(Cn)
    out = np.full(Cn.shape, np.nan)
    out[..., :-1] = np.log(a[..., :-1] / a[..., 1:])
    return out
