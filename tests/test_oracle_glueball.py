"""Pins of the glueball oracle (oracle/glueball.py) against symmetry and
closed forms: Hermitian traceless B, gauge covariance of B and D_j B and
gauge invariance of O_1..O_5, a vanishing field on unit links, the clover
of constant links written as explicit path products, the sign flip of all
five operators under spatial parity (each has an odd number of
derivatives: the "-" of A1^{-+}), their invariance under a 90-degree
rotation of the lattice (A1), and their behaviour under complex
conjugation of the links (charge conjugation)."""
import numpy as np
import pytest

from oracle import glueball as og
from paper_2609_37723_b300 import synth


def _coords(L):
    s = np.arange(L ** 3)
    return s % L, (s // L) % L, s // (L * L)


def _site(L, x, y, z):
    return (x % L) + L * ((y % L) + L * (z % L))


def _links(L, seed):
    return synth.haar_su3(np.random.default_rng(seed), (3, L ** 3))


def _gauge(U, Om, L):
    x, y, z = _coords(L)
    out = np.empty_like(U)
    for k in range(3):
        d = [int(k == 0), int(k == 1), int(k == 2)]
        nb = _site(L, x + d[0], y + d[1], z + d[2])
        out[k] = np.einsum("sab,sbc,sdc->sad", Om, U[k], Om[nb].conj())
    return out


def test_magnetic_field_hermitian_traceless():
    L = 4
    B = og.magnetic(_links(L, 1), L)
    assert np.allclose(B, np.conj(np.swapaxes(B, -1, -2)), atol=1e-13)
    assert np.allclose(np.einsum("isaa->is", B), 0, atol=1e-13)


def test_unit_links_give_zero_field_and_operators():
    L = 3
    U = np.broadcast_to(np.eye(3), (3, L ** 3, 3, 3)).astype(np.complex128)
    assert np.allclose(og.magnetic(U, L), 0)
    assert np.allclose(og.operators_t(U, L), 0)


def test_gauge_covariance_and_invariance():
    L = 4
    U = _links(L, 2)
    Om = synth.haar_su3(np.random.default_rng(3), (L ** 3,))
    U2 = _gauge(U, Om, L)
    B, B2 = og.magnetic(U, L), og.magnetic(U2, L)
    rot = lambda X: np.einsum("sab,sbc,sdc->sad", Om, X, Om.conj())
    for i in range(3):
        assert np.allclose(B2[i], rot(B[i]), atol=1e-12)
        for j in range(3):
            assert np.allclose(og.adj_deriv(U2, B2[i], L, j), rot(og.adj_deriv(U, B[i], L, j)), atol=1e-12)
    assert np.allclose(og.operators_t(U2, L), og.operators_t(U, L), atol=1e-10)


def test_constant_links_clover_closed_form():
    """Constant links M_k: the four leaves of the (mu, nu) clover are the
    path products M_mu M_nu M_mu^+ M_nu^+, M_nu M_mu^+ M_nu^+ M_mu,
    M_mu^+ M_nu^+ M_mu M_nu, M_nu^+ M_mu M_nu M_mu^+; D_j X = (M_j X M_j^+ -
    M_j^+ X M_j) / 2 for a constant X."""
    L = 3
    M = synth.haar_su3(np.random.default_rng(4), (3,))
    U = np.broadcast_to(M[:, None], (3, L ** 3, 3, 3)).copy()
    d = lambda a: a.conj().T
    for mu, nu in [(0, 1), (1, 2), (2, 0), (1, 0)]:
        a, b = M[mu], M[nu]
        Q = a @ b @ d(a) @ d(b) + b @ d(a) @ d(b) @ a + d(a) @ d(b) @ a @ b + d(b) @ a @ b @ d(a)
        F = (Q - d(Q)) / 8j
        F = F - np.trace(F) / 3 * np.eye(3)
        assert np.allclose(og.clover(U, L, mu, nu), F[None], atol=1e-13)
    X = np.random.default_rng(5).standard_normal((3, 3)) + 0j
    X = X + X.T
    Xf = np.broadcast_to(X, (L ** 3, 3, 3)).copy()
    for j in range(3):
        want = 0.5 * (M[j] @ X @ d(M[j]) - d(M[j]) @ X @ M[j])
        assert np.allclose(og.adj_deriv(U, Xf, L, j), want[None], atol=1e-13)


def _parity(U, L):
    """U'_k(x) = U_k(-x - e_k)^dagger (the link from -x to -x - e_k, reversed)."""
    x, y, z = _coords(L)
    out = np.empty_like(U)
    for k in range(3):
        d = [int(k == 0), int(k == 1), int(k == 2)]
        src = _site(L, -x - d[0], -y - d[1], -z - d[2])
        out[k] = np.conj(np.swapaxes(U[k][src], -1, -2))
    return out


def _rotate_z(U, L):
    """90 degrees about z: R(x, y, z) = (-y, x, z), so R^-1 e_x = -e_y,
    R^-1 e_y = e_x, and U'_x(x) = U_y(R^-1 x - e_y)^dagger, U'_y(x) =
    U_x(R^-1 x), U'_z(x) = U_z(R^-1 x), R^-1 (x, y, z) = (y, -x, z)."""
    x, y, z = _coords(L)
    rx, ry, rz = y, -x, z
    out = np.empty_like(U)
    out[0] = np.conj(np.swapaxes(U[1][_site(L, rx, ry - 1, rz)], -1, -2))
    out[1] = U[0][_site(L, rx, ry, rz)]
    out[2] = U[2][_site(L, rx, ry, rz)]
    return out


def test_operators_odd_under_parity():
    L = 4
    U = _links(L, 6)
    O = og.operators_t(U, L)
    assert np.all(np.abs(O) > 1e-6)
    assert np.allclose(og.operators_t(_parity(U, L), L), -O, rtol=1e-10, atol=1e-10)


def test_operators_invariant_under_cubic_rotation():
    L = 4
    U = _links(L, 7)
    O = og.operators_t(U, L)
    assert np.allclose(og.operators_t(_rotate_z(U, L), L), O, rtol=1e-10, atol=1e-10)


def test_charge_conjugation():
    """U -> U*: B -> -B*, D_j B -> -(D_j B)*: a trace of n fields becomes
    (-1)^n times the conjugate; O_2 has three fields, the others two."""
    L = 4
    U = _links(L, 8)
    O = og.operators_t(U, L)
    Oc = og.operators_t(np.conj(U), L)
    assert np.allclose(Oc, np.array([1, -1, 1, 1, 1]) * np.conj(O), rtol=1e-10, atol=1e-10)


def test_operators_brute_force_o1():
    """O_1 by loops over sites and colour indices, neighbours from
    coordinates, on a 3^3 lattice."""
    L = 3
    U = _links(L, 9)
    B = og.magnetic(U, L)
    x, y, z = _coords(L)
    d = lambda a: a.conj().T
    total = 0j
    for s in range(L ** 3):
        for i, j, k, e in og.EPS:
            dd = [int(j == 0), int(j == 1), int(j == 2)]
            sp = _site(L, x[s] + dd[0], y[s] + dd[1], z[s] + dd[2])
            sm = _site(L, x[s] - dd[0], y[s] - dd[1], z[s] - dd[2])
            DB = 0.5 * (U[j, s] @ B[k, sp] @ d(U[j, s]) - d(U[j, sm]) @ B[k, sm] @ U[j, sm])
            total += e * np.trace(B[i, s] @ DB)
    assert abs(og.operators_t(U, L)[0] - total) < 1e-10 * (1 + abs(total))


def test_summation_by_parts_relates_o4_and_o5():
    """D_j is anti-self-adjoint under sum_x Tr (periodic boundaries:
    sum_x Tr(X D_j Y) = -sum_x Tr((D_j X) Y)), and two summations by parts
    and a relabelling turn O_5 as printed into -O_4: the identity holds on
    the lattice to rounding."""
    L = 4
    U = _links(L, 10)
    O = og.operators_t(U, L)
    assert abs(O[3] + O[4]) < 1e-10 * abs(O[3])
    B = og.magnetic(U, L)
    X, Y = B[0], og.adj_deriv(U, B[1], L, 2)
    lhs = np.einsum("sab,sba->", X, og.adj_deriv(U, Y, L, 1))
    rhs = -np.einsum("sab,sba->", og.adj_deriv(U, X, L, 1), Y)
    assert abs(lhs - rhs) < 1e-10 * (1 + abs(lhs))
