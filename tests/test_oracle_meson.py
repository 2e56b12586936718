"""Pins of the meson oracle (oracle/meson.py) against facts fixed by the
mathematics rather than by its own formulas: gauge covariance, closed forms
on plane waves with unit or constant links, brute-force loops on a tiny
lattice, the backward propagator of an explicit gamma_5-hermitian inverse,
the Kronecker factorisation of the spin and mode traces, and the exact
spectrum of a rank-n correlation matrix after pruning."""
import itertools
import math

import numpy as np
import pytest

from oracle import meson, nucleon
from paper_2609_37723_b300 import synth


def _rng(seed):
    return np.random.default_rng(seed)


def _cgauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def _coords(L):
    s = np.arange(L ** 3)
    return s % L, (s // L) % L, s // (L * L)


def _site(L, x, y, z):
    return (x % L) + L * ((y % L) + L * (z % L))


def _neighbour_table(L):
    """nb[k][s][+1 / -1] by explicit coordinate arithmetic."""
    x, y, z = _coords(L)
    nb = np.zeros((3, L ** 3, 2), dtype=np.int64)
    for k in range(3):
        dx = [int(k == 0), int(k == 1), int(k == 2)]
        nb[k, :, 0] = _site(L, x + dx[0], y + dx[1], z + dx[2])
        nb[k, :, 1] = _site(L, x - dx[0], y - dx[1], z - dx[2])
    return nb


# ------------------------------------------------------------------- gammas


def test_gamma_algebra():
    """Euclidean Clifford algebra {g_mu, g_nu} = 2 delta, hermitian, g5 anticommutes."""
    gs = meson.GAMMA_K + [meson.GAMMA_4]
    for a in range(4):
        assert np.allclose(gs[a], gs[a].conj().T)
        for b in range(4):
            assert np.allclose(gs[a] @ gs[b] + gs[b] @ gs[a], 2.0 * (a == b) * np.eye(4))
        assert np.allclose(meson.GAMMA_5 @ gs[a] + gs[a] @ meson.GAMMA_5, 0)
    assert np.allclose(meson.GAMMA_5 @ meson.GAMMA_5, np.eye(4))
    assert np.allclose(meson.GAMMA_4, np.diag([1, 1, -1, -1]))


def test_links_are_su3():
    U = synth.meson_config("tiny").links(0)
    assert np.allclose(np.einsum("...ab,...cb->...ac", U, U.conj()), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)


# -------------------------------------------------------------- derivatives


def _gauge_transform(U, f, Om, L):
    """U_k(x) -> Om(x) U_k(x) Om(x+k)^dagger, f(x) -> Om(x) f(x)."""
    nb = _neighbour_table(L)
    U2 = np.empty_like(U)
    for k in range(3):
        U2[k] = np.einsum("sab,sbc,sdc->sad", Om, U[k], Om[nb[k, :, 0]].conj())
    f2 = np.einsum("sab,nsb->nsa", Om, f)
    return U2, f2


def test_derivatives_gauge_covariant():
    L = 4
    rng = np.random.default_rng(5)
    U = synth.haar_su3(rng, (3, L ** 3))
    f = _cgauss(rng, (3, L ** 3, 3))
    Om = synth.haar_su3(rng, (L ** 3,))
    U2, f2 = _gauge_transform(U, f, Om, L)
    for k in range(3):
        got = meson.nabla(U2, f2, L, k)
        assert np.allclose(got, np.einsum("sab,nsb->nsa", Om, meson.nabla(U, f, L, k)), atol=1e-12)
        got = meson.bb(U2, f2, L, k)
        assert np.allclose(got, np.einsum("sab,nsb->nsa", Om, meson.bb(U, f, L, k)), atol=1e-12)


def test_elementals_gauge_invariant():
    L = 4
    rng = np.random.default_rng(6)
    U = synth.haar_su3(rng, (3, L ** 3))
    v = _cgauss(rng, (5, L ** 3, 3))
    Om = synth.haar_su3(rng, (L ** 3,))
    U2, v2 = _gauge_transform(U, v, Om, L)
    mom = np.array([[0, 0, 0], [1, 0, 2]])
    a = meson.elementals_t(v, U, L, mom)
    b = meson.elementals_t(v2, U2, L, mom)
    assert np.allclose(a, b, atol=1e-11)


def test_plane_wave_unit_links():
    """U = 1: nabla_k e^{iqx} c = i sin(theta_k) e^{iqx} c, BB = 0."""
    L = 6
    x, y, z = _coords(L)
    n = np.array([1, 2, -1])
    th = 2 * np.pi * n / L
    rng = np.random.default_rng(7)
    c = _cgauss(rng, 3)
    f = (np.exp(1j * (th[0] * x + th[1] * y + th[2] * z))[:, None] * c[None, :])[None]
    U = np.broadcast_to(np.eye(3), (3, L ** 3, 3, 3)).astype(np.complex128)
    for k in range(3):
        assert np.allclose(meson.nabla(U, f, L, k), 1j * math.sin(th[k]) * f, atol=1e-13)
        assert np.allclose(meson.bb(U, f, L, k), 0, atol=1e-13)


def test_constant_links_closed_form():
    """U_k(x) = M_k: on e^{iqx} c, nabla_k acts as D_k = (e^{i th_k} M_k -
    e^{-i th_k} M_k^dagger) / 2 and BB_i as the commutator [D_j, D_k]."""
    L = 5
    x, y, z = _coords(L)
    n = np.array([2, 0, 1])
    th = 2 * np.pi * n / L
    rng = np.random.default_rng(8)
    M = synth.haar_su3(rng, (3,))
    U = np.broadcast_to(M[:, None], (3, L ** 3, 3, 3)).copy()
    c = _cgauss(rng, 3)
    wave = np.exp(1j * (th[0] * x + th[1] * y + th[2] * z))
    f = (wave[:, None] * c[None, :])[None]
    D = [0.5 * (np.exp(1j * th[k]) * M[k] - np.exp(-1j * th[k]) * M[k].conj().T) for k in range(3)]
    for k in range(3):
        want = wave[:, None] * (D[k] @ c)[None, :]
        assert np.allclose(meson.nabla(U, f, L, k)[0], want, atol=1e-13)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        want = wave[:, None] * ((D[j] @ D[k] - D[k] @ D[j]) @ c)[None, :]
        assert np.allclose(meson.bb(U, f, L, i)[0], want, atol=1e-12)


def test_elementals_constant_links_closed_form():
    """Plane-wave vectors v_i = e^{i q_i x} c_i with constant links: Phi^d_ij(p)
    = V3 delta(q_j - q_i = p mod L) c_i^dagger X_d(q_j) c_j, X_0 = 1,
    X_(1+k) = D_k, X_(4+i) = [D_j, D_k]."""
    L = 4
    x, y, z = _coords(L)
    rng = np.random.default_rng(9)
    M = synth.haar_su3(rng, (3,))
    U = np.broadcast_to(M[:, None], (3, L ** 3, 3, 3)).copy()
    qs = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 3], [1, 0, 1]])
    cs = _cgauss(rng, (len(qs), 3))
    v = np.stack([np.exp(2j * np.pi * (q[0] * x + q[1] * y + q[2] * z) / L)[:, None] * c[None, :]
                  for q, c in zip(qs, cs)])
    mom = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 3], [-1, 1, 2]])
    phi = meson.elementals_t(v, U, L, mom)
    V3 = L ** 3
    for qi, p in enumerate(mom):
        for i, j in itertools.product(range(len(qs)), repeat=2):
            th = 2 * np.pi * qs[j] / L
            D = [0.5 * (np.exp(1j * th[k]) * M[k] - np.exp(-1j * th[k]) * M[k].conj().T) for k in range(3)]
            X = [np.eye(3)] + D + [D[(a + 1) % 3] @ D[(a + 2) % 3] - D[(a + 2) % 3] @ D[(a + 1) % 3]
                                   for a in range(3)]
            match = np.all((qs[j] - qs[i] - p) % L == 0)
            for d in range(7):
                want = V3 * (cs[i].conj() @ X[d] @ cs[j]) if match else 0.0
                assert abs(phi[qi, d, i, j] - want) < 1e-10 * V3


def test_elementals_brute_force_loops():
    """Element-by-element loops over sites and colours with neighbours from
    coordinate arithmetic (independent of the array shifts)."""
    L = 3
    rng = np.random.default_rng(10)
    U = synth.haar_su3(rng, (3, L ** 3))
    v = _cgauss(rng, (3, L ** 3, 3))
    nb = _neighbour_table(L)
    x, y, z = _coords(L)
    p = np.array([1, 2, 0])
    phase = np.exp(-2j * np.pi * (p[0] * x + p[1] * y + p[2] * z) / L)

    def nab(f, k):  # f[s][a]
        out = np.zeros_like(f)
        for s in range(L ** 3):
            sp, sm = nb[k, s, 0], nb[k, s, 1]
            for a in range(3):
                acc = 0
                for b in range(3):
                    acc += U[k, s, a, b] * f[sp, b] - np.conj(U[k, sm, b, a]) * f[sm, b]
                out[s, a] = 0.5 * acc
        return out

    phi = meson.elementals_t(v, U, L, p[None])
    for i, j in [(0, 1), (2, 2), (1, 0)]:
        fields = [v[j]] + [nab(v[j], k) for k in range(3)]
        fields += [nab(nab(v[j], (a + 2) % 3), (a + 1) % 3) - nab(nab(v[j], (a + 1) % 3), (a + 2) % 3)
                   for a in range(3)]
        for d, F in enumerate(fields):
            want = sum(phase[s] * np.conj(v[i, s, a]) * F[s, a] for s in range(L ** 3) for a in range(3))
            assert abs(phi[0, d, i, j] - want) < 1e-12


# -------------------------------------------------------------- correlator


def _random_phi(rng, npm, nv):
    return _cgauss(rng, (npm, 7, nv, nv))


def test_backward_propagator_from_explicit_inverse():
    """tau(t,0) and tau(0,t) as blocks of the inverse of a gamma_5-hermitian
    matrix (built from its own gamma_5 up to sign): the correlator from the
    forward block alone equals -Tr[Phi_a S(t,0) Phibar_b S(0,t)] with S(0,t)
    read off the inverse."""
    nv = 3
    rng = np.random.default_rng(11)
    g5 = np.kron(np.array([[0, 1], [1, 0]]), np.eye(2))  # gamma_5 up to sign
    G5 = np.kron(np.eye(2), np.kron(g5, np.eye(nv)))     # two timeslices
    H = _cgauss(rng, (8 * nv, 8 * nv))
    H = H + H.conj().T + 12 * np.eye(8 * nv)
    S = np.linalg.inv(G5 @ H)
    assert np.allclose(G5 @ S @ G5, S.conj().T, atol=1e-12)
    n4 = 4 * nv
    S_t0, S_0t = S[n4:, :n4], S[:n4, n4:]
    phi_t = _random_phi(rng, 1, nv)
    phi_0 = _random_phi(rng, 1, nv)
    prof = np.stack([np.linspace(1, 0.3, nv), np.ones(nv)])
    C = meson.correlator_t(phi_t, phi_0, S_t0, prof)
    for typ_a, typ_b in itertools.product(range(3), repeat=2):
        for sa, sb in itertools.product(range(2), repeat=2):
            A = meson.sink_matrix(phi_t[0], prof[sa], typ_a)
            B = meson.source_matrix(phi_0[0], prof[sb], typ_b)
            want = -np.trace(A @ S_t0 @ B @ S_0t)
            assert abs(C[0, 2 * typ_a + sa, 2 * typ_b + sb] - want) < 1e-11 * (1 + abs(want))


def test_source_matrix_is_operator_adjoint():
    """O = qbar M q = psi^dagger (gamma_4 M) psi: the creation operator
    O^dagger has the matrix N with gamma_4 N = (gamma_4 M)^dagger."""
    nv = 3
    rng = np.random.default_rng(12)
    phi = _random_phi(rng, 1, nv)[0]
    g = rng.uniform(0.2, 1.0, nv)
    G4 = np.kron(meson.GAMMA_4, np.eye(nv))
    for typ in range(3):
        M = meson.sink_matrix(phi, g, typ)
        N = meson.source_matrix(phi, g, typ)
        assert np.allclose(G4 @ N, (G4 @ M).conj().T, atol=1e-13)


def test_correlator_kronecker_factorisation():
    """tau = S (x) T: the trace factorises into a 4 x 4 spin trace and an
    N_v x N_v mode trace per pair of operator terms."""
    nv = 4
    rng = np.random.default_rng(13)
    S4 = _cgauss(rng, (4, 4))
    T = _cgauss(rng, (nv, nv))
    tau = np.kron(S4, T)
    phi_t = _random_phi(rng, 1, nv)
    phi_0 = _random_phi(rng, 1, nv)
    prof = np.stack([np.linspace(1, 0.1, nv)])
    C = meson.correlator_t(phi_t, phi_0, tau, prof)
    g = prof[0]
    g5 = meson.GAMMA_5
    for ta, tb in itertools.product(range(3), repeat=2):
        want = 0
        for (da, Ga), (db, Gb) in itertools.product(meson.operator_terms(ta), meson.operator_terms(tb)):
            Gbar = meson.GAMMA_4 @ Gb.conj().T @ meson.GAMMA_4
            spin = np.trace(Ga @ S4 @ Gbar @ g5 @ S4.conj().T @ g5)
            A = g[:, None] * phi_t[0, da] * g[None, :]
            B = (g[:, None] * phi_0[0, db] * g[None, :]).conj().T
            mode = np.trace(A @ T @ B @ T.conj().T)
            want += spin * mode
        assert abs(C[0, ta, tb] + want) < 1e-11 * (1 + abs(want))


def test_unit_propagator_reduces_to_gamma_traces():
    """tau = 1: C_ab = -Tr_spin[Gamma_a gamma_4 Gamma_b^dagger gamma_4] Tr[A B^dagger];
    for type 0 with itself the spin trace is -4 (gamma_4 gamma_5 squared
    conjugated by gamma_4), so C = 4 ||g Phi^0 g||_F^2 > 0."""
    nv = 5
    rng = np.random.default_rng(14)
    phi = _random_phi(rng, 1, nv)
    prof = np.stack([np.linspace(1, 0.2, nv)])
    C = meson.correlator_t(phi, phi, np.eye(4 * nv), prof)
    A = prof[0][:, None] * phi[0, 0] * prof[0][None, :]
    assert abs(C[0, 0, 0] - 4 * np.linalg.norm(A) ** 2) < 1e-11 * np.linalg.norm(A) ** 2


def test_exponential_decay_of_scaled_perambulator():
    """tau(t) = e^{-m t} T gives C(t) = e^{-2 m t} C(0) exactly."""
    nv = 3
    rng = np.random.default_rng(15)
    T = _cgauss(rng, (4 * nv, 4 * nv))
    phi = _random_phi(rng, 1, nv)
    prof = np.stack([np.ones(nv), np.linspace(1, 0.5, nv)])
    c0 = meson.correlator_t(phi, phi, T, prof)
    c3 = meson.correlator_t(phi, phi, math.exp(-0.7 * 3) * T, prof)
    assert np.allclose(c3, math.exp(-1.4 * 3) * c0, rtol=1e-12, atol=0)


# ------------------------------------------------------------ pruning, GEVP


def test_prune_rank_n_spectrum_exact():
    """C(t) = Z diag(lambda^t) Z^dagger of rank n = 8 in 21 dimensions: the
    pruned 8 x 8 GEVP returns lambda_n^(t - t0) exactly."""
    rng = np.random.default_rng(16)
    nops, n, nt = 21, 8, 6
    Z = _cgauss(rng, (nops, n))
    lam = np.sort(rng.uniform(0.2, 0.9, n))[::-1]
    C = np.stack([Z @ np.diag(lam ** t) @ Z.conj().T for t in range(nt)], axis=-1)[None]
    Ct, Un, sv = meson.prune(C, 1, n)
    assert np.allclose(Un[0].conj().T @ Un[0], np.eye(n), atol=1e-12)
    assert np.all(np.diff(sv[0]) <= 0)
    assert np.all(sv[0, n:] < 1e-10 * sv[0, 0])
    ev = meson.gevp(Ct, 0)
    for t in range(nt):
        got = np.sort(ev[0, t].real)[::-1]
        assert np.allclose(got, lam ** t, rtol=1e-9, atol=0)
        assert np.allclose(ev[0, t].imag, 0, atol=1e-9)


def test_prune_hermitian_diagonalises_at_t_prune():
    rng = np.random.default_rng(17)
    A = _cgauss(rng, (21, 21))
    H = A @ A.conj().T
    C = np.stack([H, H @ H], axis=-1)[None]
    Ct, Un, sv = meson.prune(C, 0, 8)
    assert np.allclose(Ct[0, :, :, 0], np.diag(sv[0, :8]), atol=1e-10 * sv[0, 0])
    assert np.allclose(Ct[0, :, :, 1], np.diag(sv[0, :8] ** 2), atol=1e-10 * sv[0, 0] ** 2)


def test_prune_all_keeps_gevp():
    rng = np.random.default_rng(18)
    C = _cgauss(rng, (1, 21, 21, 3))
    Ct, _, _ = meson.prune(C, 1, 21)
    assert np.allclose(meson.gevp(Ct, 0), nucleon.gevp(C, 0), rtol=1e-8, atol=1e-10)


def test_oracle_tiny_workload_shapes():
    m = synth.meson_config("tiny")
    v, U, tau = m.all_eigvecs(), m.all_links(), m.all_perambulators()
    phi = meson.elementals(v, U, m.L, m.mom)
    assert phi.shape == (m.nt, m.np_, 7, m.nv, m.nv)
    C = meson.correlator(phi, phi[0], tau, m.prof)
    assert C.shape == (m.np_, 21, 21, m.nt)
    Ct, _, _ = meson.prune(C, m.t_prune, m.nkeep)
    assert Ct.shape == (m.np_, 8, 8, m.nt)
    assert np.all(np.isfinite(meson.gevp(Ct, 0)))
