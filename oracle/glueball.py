"""FP64 CPU oracle for the A1^{-+} glueball operators built from the
chromo-magnetic field and adjoint covariant derivatives.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.  It shares no
code with the CUDA library: a plain restatement of the definitions in
complex128.

What it computes (paper Sec. 2.2, "Improved glueball operators": the
chromo-magnetic component B_i = eps_ijk F_jk of the field strength in the
clover discretisation, adjoint spatial gauge-covariant symmetric
differences D_j, and the five A1^{-+} operators O_1 .. O_5):

* clover field strength in the spatial plane (mu, nu) at site x, from the
  four plaquettes of the plane that start and end at x (counter-clockwise
  in (mu, nu)):
      Q = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        + U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
        + U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
        + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
      F_{mu nu} = (Q - Q^dag) / (8 i), minus a third of its trace
  (Hermitian and traceless; lattice units);
* B_i = eps_ijk F_jk = 2 F_jk for (i, j, k) cyclic;
* adjoint covariant symmetric difference of a matrix field X,
      (D_j X)(x) = 1/2 [U_j(x) X(x+j) U_j(x)^dag - U_j(x-j)^dag X(x-j) U_j(x-j)],
  powers D_j^2 = D_j D_j applied right to left;
* the operators, repeated indices summed (eps the Levi-Civita symbol):
      O_1 = sum_x Tr(eps_ijk B_i D_j B_k)
      O_2 = sum_x Tr(eps_ijk eps_ilm B_j B_k D_l B_m)
      O_3 = sum_x Tr(eps_ijk B_i D_j^3 B_k)
      O_4 = sum_x Tr(eps_ijk B_i D_j^2 D_k B_j)
      O_5 = sum_x Tr(eps_ijk B_i D_j D_i^2 B_k)
  at zero momentum, one complex number per operator and timeslice.

Layouts shared with the library's C interface (inputs and outputs only):
links U[t][k][s][a][b] (direction k = x, y, z; s = x + L(y + Lz)); operators
O[t][n], n = 0..4.
"""
from __future__ import annotations

import itertools

import numpy as np

N_OPS = 5


def _eps(i, j, k) -> int:
    return int(np.sign((j - i) * (k - i) * (k - j)))


EPS = [(i, j, k, _eps(i, j, k)) for i, j, k in itertools.permutations(range(3))]


def _shift(f: np.ndarray, L: int, k: int, step: int) -> np.ndarray:
    """g(x) = f(x + step e_k) for a site field f[V3][3][3]."""
    g = f.reshape(L, L, L, 3, 3)
    return np.roll(g, -step, axis=2 - k).reshape(f.shape)


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum("sab,sbc->sac", out, m)
    return out


def clover(U_t: np.ndarray, L: int, mu: int, nu: int) -> np.ndarray:
    """F_{mu nu}(x) [V3][3][3], Hermitian and traceless."""
    U = [np.asarray(U_t[k], dtype=np.complex128) for k in range(3)]
    Um, Un = U[mu], U[nu]
    sh = lambda f, k, st: _shift(f, L, k, st)
    q = _mm(Um, sh(Un, mu, 1), _dag(sh(Um, nu, 1)), _dag(Un))
    q = q + _mm(Un, _dag(sh(sh(Um, mu, -1), nu, 1)), _dag(sh(Un, mu, -1)), sh(Um, mu, -1))
    q = q + _mm(_dag(sh(Um, mu, -1)), _dag(sh(sh(Un, mu, -1), nu, -1)), sh(sh(Um, mu, -1), nu, -1), sh(Un, nu, -1))
    q = q + _mm(_dag(sh(Un, nu, -1)), sh(Um, nu, -1), sh(sh(Un, mu, 1), nu, -1), _dag(Um))
    F = (q - _dag(q)) / 8j
    tr = np.einsum("saa->s", F) / 3.0
    return F - tr[:, None, None] * np.eye(3)


def magnetic(U_t: np.ndarray, L: int) -> np.ndarray:
    """B_i(x) = eps_ijk F_jk(x) = 2 F_jk for (i, j, k) cyclic: [3][V3][3][3]."""
    return np.stack([2.0 * clover(U_t, L, (i + 1) % 3, (i + 2) % 3) for i in range(3)])


def adj_deriv(U_t: np.ndarray, X: np.ndarray, L: int, j: int) -> np.ndarray:
    """(D_j X)(x) = 1/2 [U_j(x) X(x+j) U_j(x)^dag - U_j(x-j)^dag X(x-j) U_j(x-j)]."""
    Uj = np.asarray(U_t[j], dtype=np.complex128)
    Ub = _shift(Uj, L, j, -1)
    fwd = _mm(Uj, _shift(X, L, j, 1), _dag(Uj))
    bwd = _mm(_dag(Ub), _shift(X, L, j, -1), Ub)
    return 0.5 * (fwd - bwd)


def _tr(*ms) -> complex:
    """sum_x Tr(m1 m2 ...)."""
    return complex(np.einsum("saa->", _mm(*ms)))


def operators_t(U_t: np.ndarray, L: int) -> np.ndarray:
    """O_1 .. O_5 of one timeslice: complex [5]."""
    B = magnetic(U_t, L)
    D = lambda X, j: adj_deriv(U_t, X, L, j)
    O = np.zeros(N_OPS, dtype=np.complex128)
    for i, j, k, e in EPS:
        O[0] += e * _tr(B[i], D(B[k], j))
        O[2] += e * _tr(B[i], D(D(D(B[k], j), j), j))
        O[3] += e * _tr(B[i], D(D(D(B[j], k), j), j))
        O[4] += e * _tr(B[i], D(D(D(B[k], i), i), j))
    for (i, j, k, e1), (i2, l, m, e2) in itertools.product(EPS, EPS):
        if i == i2:
            O[1] += e1 * e2 * _tr(B[j], B[k], D(B[m], l))
    return O


def operators(U: np.ndarray, L: int) -> np.ndarray:
    """O[t][n] for every timeslice of U[t][3][V3][3][3]."""
    return np.stack([operators_t(U[t], L) for t in range(U.shape[0])])
