"""Pins of the oracle's N_B x N_B correlation matrix and GEVP (CPU only).

The correlation matrix of the profiled elementals Phi^(a) = g g g Phi
(Sec. 2.1, displayed equation; "compute an N_B x N_B correlation matrix and
solve a GEVP").  The spin and Wick structure the paper leaves out is the
positive-parity nucleon with C gamma_5 diquark and u<->u exchange (module
docstring of the oracle).
"""
import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth


def rand_packed(rng, nv, lead=()):
    return synth.complex_gaussian(rng, lead + (orc.n_triples(nv),))


def psi(G, mu):
    """Psi^mu_{(alpha i)(beta j)(gamma k)} = G_ijk Gamma_{alpha beta} delta_{gamma mu}."""
    nv = G.shape[0]
    e = np.zeros(4)
    e[mu] = 1
    return np.einsum("ijk,ab,c->aibjck", G, orc.GAMMA, e).reshape(4 * nv, 4 * nv, 4 * nv)


def brute_C(phi_snk, phi_src, tau, g_snk, g_src):
    """Six-index sum with the direct and the exchange term written separately."""
    nv = tau.shape[0] // 4
    nb = g_snk.shape[0]
    ds, d0 = orc.unpack(phi_snk, nv), orc.unpack(phi_src, nv)
    C = np.zeros((nb, nb), dtype=np.complex128)
    for a in range(nb):
        for b in range(nb):
            Ga = ds * np.einsum("i,j,k->ijk", g_snk[a], g_snk[a], g_snk[a])
            Gb = d0 * np.einsum("i,j,k->ijk", g_src[b], g_src[b], g_src[b])
            for mu in range(4):
                for nu in range(4):
                    if orc.P_PLUS[nu, mu] == 0:
                        continue
                    snk = psi(Ga, mu)
                    src = psi(Gb, nu)
                    bracket = src - src.transpose(2, 1, 0)      # direct - exchange
                    C[a, b] += orc.P_PLUS[nu, mu] * np.einsum(
                        "IJK,IL,JM,KN,LMN->", snk, tau, tau, tau, np.conj(bracket), optimize="optimal")
    return C


def rand_case(seed, nv, nb=2):
    rng = np.random.default_rng(seed)
    phs = rand_packed(rng, nv)
    ph0 = rand_packed(rng, nv)
    tau = synth.complex_gaussian(rng, (4 * nv, 4 * nv))
    g_snk = rng.uniform(0.2, 1.0, size=(nb, nv))
    g_src = rng.uniform(0.2, 1.0, size=(nb, nv))
    return phs, ph0, tau, g_snk, g_src


@pytest.mark.parametrize("nv,seed", [(3, 1), (4, 2), (5, 3)])
def test_brute_force_unfolded_wick(nv, seed):
    phs, ph0, tau, gs, g0 = rand_case(seed, nv)
    got = orc.correlator_tp(phs, ph0, tau, gs, g0)
    ref = brute_C(phs, ph0, tau, gs, g0)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * scale)


def test_planted_mistakes_are_caught(monkeypatch):
    """Dropping the exchange term, flipping its sign, flipping the sign of one
    2x2 block of Gamma or using the negative-parity projector in the oracle
    must each break agreement with the brute force.  (Transposing Gamma is
    not a detectable mistake: Gamma^T = -Gamma enters sink and source once
    each, so the overall sign cancels.)"""
    phs, ph0, tau, gs, g0 = rand_case(7, 4)
    ref = brute_C(phs, ph0, tau, gs, g0)
    good = orc.source_spin

    def direct_only(nu):
        return {k: v for k, v in ((k, orc.GAMMA[k[0], k[1]] * (k[2] == nu)) for k in good(nu)) if v != 0}

    def flipped(nu):
        s = {}
        for a in range(4):
            for b in range(4):
                for c in range(4):
                    val = orc.GAMMA[a, b] * (c == nu) - orc.GAMMA[c, b] * (a == nu)
                    if val:
                        s[(a, b, c)] = val
        return s

    for bad in (direct_only, flipped):
        monkeypatch.setattr(orc, "source_spin", bad)
        wrong = orc.correlator_tp(phs, ph0, tau, gs, g0)
        assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()
    monkeypatch.setattr(orc, "source_spin", good)
    g2 = orc.GAMMA.copy()
    g2[2:, 2:] *= -1
    monkeypatch.setattr(orc, "GAMMA", g2)
    wrong = orc.correlator_tp(phs, ph0, tau, gs, g0)
    assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()
    monkeypatch.setattr(orc, "GAMMA", orc.GAMMA)
    monkeypatch.undo()
    monkeypatch.setattr(orc, "P_PLUS", np.diag([0.0, 0.0, 1.0, 1.0]))
    wrong = orc.correlator_tp(phs, ph0, tau, gs, g0)
    assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()


def test_folded_spin_tensor_counts():
    """Seven distinct source spin triples per nu; the triples hit by both
    Wick terms carry weight -2 (nu = 0) and +2 (nu = 1)."""
    s0, s1 = orc.source_spin(0), orc.source_spin(1)
    assert len(s0) == 7 and len(s1) == 7
    assert s0[(0, 1, 0)] == -2 and s1[(1, 0, 1)] == 2
    assert sorted(abs(x) for x in s0.values()) == [1, 1, 1, 1, 1, 1, 2]


def test_identity_perambulator_closed_form():
    """tau = 1 (spin (x) mode): C_ab = kappa sum_ijk Phi^(a)snk Phi^(b)src*,
    kappa = sum_mu [||Gamma||_F^2 + sum_beta Gamma_{mu beta}^2] = 2*(4+1) = 10."""
    nv = 5
    rng = np.random.default_rng(23)
    phs, ph0 = rand_packed(rng, nv), rand_packed(rng, nv)
    g = synth.gaussian_profiles(nv, [0.3, 0.7, 1.5])
    tau = np.eye(4 * nv)
    got = orc.correlator_tp(phs, ph0, tau, g, g)
    ds, d0 = orc.unpack(phs, nv), orc.unpack(ph0, nv)
    for a in range(3):
        for b in range(3):
            Ga = orc.profile_scale(ds, g[a])
            Gb = orc.profile_scale(d0, g[b])
            assert abs(got[a, b] - 10.0 * np.sum(Ga * np.conj(Gb))) < 1e-12 * abs(got[a, b])


def test_rank_one_perambulator_factorises():
    """tau_{II'} = x_I y_I' splits C into multilinear evaluations of the sink
    at x and of the source bracket at y."""
    nv = 4
    rng = np.random.default_rng(29)
    phs, ph0 = rand_packed(rng, nv), rand_packed(rng, nv)
    g = rng.uniform(0.3, 1, size=(2, nv))
    x = synth.complex_gaussian(rng, 4 * nv)
    y = synth.complex_gaussian(rng, 4 * nv)
    tau = np.outer(x, y)
    got = orc.correlator_tp(phs, ph0, tau, g, g)
    ds, d0 = orc.unpack(phs, nv), orc.unpack(ph0, nv)
    for a in range(2):
        for b in range(2):
            ref = 0
            for mu in (0, 1):
                snk = psi(orc.profile_scale(ds, g[a]), mu)
                src = psi(orc.profile_scale(d0, g[b]), mu)
                br = np.conj(src - src.transpose(2, 1, 0))
                ref += np.einsum("IJK,I,J,K->", snk, x, x, x) * np.einsum("IJK,I,J,K->", br, y, y, y)
            assert abs(got[a, b] - ref) < 1e-12 * max(1.0, abs(ref))


def test_hermitian_and_positive():
    """Hermitian tau with equal sink and source elementals gives Hermitian C;
    Hermitian positive-definite tau gives positive semi-definite C."""
    nv = 4
    rng = np.random.default_rng(31)
    ph = rand_packed(rng, nv)
    g = synth.gaussian_profiles(nv, [0.3, 0.6, 1.0, 2.0])
    h = synth.complex_gaussian(rng, (4 * nv, 4 * nv))
    herm = h + h.conj().T
    C = orc.correlator_tp(ph, ph, herm, g, g)
    np.testing.assert_allclose(C, C.conj().T, atol=1e-12 * np.abs(C).max())
    hpd = h @ h.conj().T + 0.1 * np.eye(4 * nv)
    C = orc.correlator_tp(ph, ph, hpd, g, g)
    np.testing.assert_allclose(C, C.conj().T, atol=1e-12 * np.abs(C).max())
    ev = np.linalg.eigvalsh(0.5 * (C + C.conj().T))
    assert ev.min() > -1e-12 * ev.max()
    assert ev.max() > 0


def test_mode_basis_rotation():
    """v -> v W (W unitary) and tau -> (1 (x) W)^dag tau (1 (x) W) leave C
    unchanged for unit profiles; a diagonal W leaves it unchanged with any
    profiles."""
    nv = 4
    rng = np.random.default_rng(37)
    phs, ph0, tau, _, _ = rand_case(41, nv)
    W, _ = np.linalg.qr(synth.complex_gaussian(rng, (nv, nv)))

    def rot(packed, W):
        d = orc.unpack(packed, nv)
        d2 = np.einsum("ai,bj,ck,abc->ijk", W, W, W, d)
        i, j, k = orc.triples(nv)
        return d2[i, j, k]

    big = np.kron(np.eye(4), W)
    tau2 = big.conj().T @ tau @ big
    ones = np.ones((1, nv))
    c1 = orc.correlator_tp(phs, ph0, tau, ones, ones)
    c2 = orc.correlator_tp(rot(phs, W), rot(ph0, W), tau2, ones, ones)
    np.testing.assert_allclose(c2, c1, atol=1e-12 * np.abs(c1).max())
    D = np.diag(np.exp(1j * rng.uniform(0, 6.28, nv)))
    g = rng.uniform(0.2, 1, size=(3, nv))
    bigd = np.kron(np.eye(4), D)
    c1 = orc.correlator_tp(phs, ph0, tau, g, g)
    c2 = orc.correlator_tp(rot(phs, D), rot(ph0, D), bigd.conj().T @ tau @ bigd, g, g)
    np.testing.assert_allclose(c2, c1, atol=1e-12 * np.abs(c1).max())


def test_cubic_scaling_and_unit_profiles():
    phs, ph0, tau, gs, g0 = rand_case(43, 4, nb=3)
    c1 = orc.correlator_tp(phs, ph0, tau, gs, g0)
    c2 = orc.correlator_tp(phs, ph0, 0.5 * tau, gs, g0)
    np.testing.assert_allclose(c2, 0.125 * c1, atol=1e-14 * np.abs(c1).max())
    ones = np.ones((3, 4))
    cu = orc.correlator_tp(phs, ph0, tau, ones, ones)
    np.testing.assert_allclose(cu, cu[0, 0] * np.ones((3, 3)), atol=1e-13 * abs(cu[0, 0]))


def test_profile_is_diagonal_rescaling():
    """A profile that is one on a single mode isolates the triples that
    contain only that mode -- none, since i<j<k: C vanishes; two modes on,
    also none; three modes on gives one triple."""
    nv = 5
    phs, ph0, tau, _, _ = rand_case(47, nv)
    for on in ([2], [1, 3]):
        g = np.zeros((1, nv))
        g[0, on] = 1
        assert abs(orc.correlator_tp(phs, ph0, tau, g, g)[0, 0]) < 1e-300
    g = np.zeros((1, nv))
    g[0, [0, 2, 4]] = 1
    keep = np.zeros(orc.n_triples(nv))
    keep[orc.triple_rank(0, 2, 4)] = 1
    a = orc.correlator_tp(phs, ph0, tau, g, g)
    b = orc.correlator_tp(phs * keep, ph0 * keep, tau, np.ones((1, nv)), np.ones((1, nv)))
    np.testing.assert_allclose(a, b, atol=1e-14 * abs(b[0, 0]))


def _per_t_case(seed, nv=4, nt=3, nb=3):
    rng = np.random.default_rng(seed)
    phs = rand_packed(rng, nv, (nt, 2))
    ph0 = rand_packed(rng, nv, (2,))
    tau = synth.complex_gaussian(rng, (nt, 4 * nv, 4 * nv))
    g = rng.uniform(0.2, 1.0, size=(nb, nv))
    return phs, ph0, tau, g


def test_per_t_profiles_equal_reproduce_fixed_profiles():
    """Profiles that depend on t (Sec. 2.1 writes g_i^(a)[t]) but are equal on
    every timeslice give the t-independent correlation matrix."""
    phs, ph0, tau, g = _per_t_case(61)
    nt = tau.shape[0]
    fixed = orc.correlator(phs, ph0, tau, g)
    per_t = orc.correlator(phs, ph0, tau, np.stack([g] * nt), prof_per_t=True)
    np.testing.assert_array_equal(per_t, fixed)


def test_per_t_profiles_sink_at_t_source_at_t0():
    """The sink elemental at t carries g[t], the source at t0 = 0 carries g[0]
    (Sec. 2.1: Phi^(a)[p,t] = g[t] g[t] g[t] Phi[p,t]).  C is cubic in each
    profile (one factor per quark), so with g[t] = c_a g for t >= 1 and
    g[0] = g, row a of C(t >= 1) scales by c_a^3 (sink side only; were g[t]
    used on both sides it would scale by c_a^3 c_b^3, were g[0] used for the
    sink not at all), while C(t = 0), where sink and source both use g[0],
    is unchanged.  Scaling the source profile g[0] instead scales the
    columns of C(t >= 1) by c_b^3 and C(0) by c_a^3 c_b^3."""
    phs, ph0, tau, g = _per_t_case(67)
    nt, nb = tau.shape[0], g.shape[0]
    c = np.array([2.0, 0.5, 1.5])
    fixed = orc.correlator(phs, ph0, tau, g)
    sink_scaled = np.stack([g] + [c[:, None] * g] * (nt - 1))
    got = orc.correlator(phs, ph0, tau, sink_scaled, prof_per_t=True)
    np.testing.assert_allclose(got[..., 0], fixed[..., 0], rtol=1e-13)
    rows = (c ** 3)[None, :, None, None]
    np.testing.assert_allclose(got[..., 1:], rows * fixed[..., 1:], rtol=1e-12)
    src_scaled = np.stack([c[:, None] * g] + [g] * (nt - 1))
    got = orc.correlator(phs, ph0, tau, src_scaled, prof_per_t=True)
    cols = (c ** 3)[None, None, :, None]
    np.testing.assert_allclose(got[..., 1:], cols * fixed[..., 1:], rtol=1e-12)
    np.testing.assert_allclose(got[..., 0], (c ** 3)[None, :, None] * (c ** 3)[None, None, :] * fixed[..., 0],
                               rtol=1e-12)
    assert nb == len(c)


# --------------------------------------------------------------------- GEVP

def test_gevp_constructed_pencil():
    """C(t) = A diag(lambda^t) B has generalized eigenvalues lambda^(t - t0)."""
    rng = np.random.default_rng(53)
    nb, nt, t0 = 5, 8, 2
    lam = np.sort(rng.uniform(0.2, 0.95, nb))[::-1]
    A = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
    B = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
    C = np.zeros((2, nb, nb, nt), dtype=np.complex128)
    for t in range(nt):
        C[0, :, :, t] = A @ np.diag(lam ** t) @ B
        C[1, :, :, t] = A @ np.diag(lam ** t) @ A.conj().T          # Hermitian pencil
    got = orc.gevp(C, t0)
    for t in range(nt):
        expect = np.sort(lam ** (t - t0))[::-1]
        np.testing.assert_allclose(got[0, t], expect, rtol=1e-9)
        np.testing.assert_allclose(got[1, t], expect, rtol=1e-9)


def _hermitian_pencil(seed, nb=5, nt=8):
    """C(t) = B^H diag(lambda^t) B: the GEVP C(t) u = lambda C(t0) u has the
    eigenvalues lambda_n^(t - t0) and the eigenvectors B^{-1} e_n (exactly)."""
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(0.2, 0.95, nb))[::-1]
    B = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
    C = np.zeros((1, nb, nb, nt), dtype=np.complex128)
    for t in range(nt):
        C[0, :, :, t] = B.conj().T @ np.diag(lam ** t) @ B
    return lam, B, C


def test_gevp_vectors_constructed_pencil():
    lam, B, C = _hermitian_pencil(71)
    nb, nt, t0 = len(lam), C.shape[-1], 2
    got_l, got_u = orc.gevp_vectors(C, t0)
    Binv = np.linalg.inv(B)
    for t in range(nt):
        if t == t0:
            continue      # every eigenvalue is 1 there: the vectors are not unique
        order = np.argsort(-(lam ** (t - t0)), kind="stable")   # t < t0 reverses the order
        np.testing.assert_allclose(got_l[0, t], (lam ** (t - t0))[order], rtol=1e-9)
        for n in range(nb):
            ref = Binv[:, order[n]] / np.linalg.norm(Binv[:, order[n]])
            u = got_u[0, t, n]
            assert abs(np.linalg.norm(u) - 1) < 1e-12
            k = np.argmax(np.abs(u))
            assert abs(u[k].imag) < 1e-14 and u[k].real > 0
            assert abs(abs(np.vdot(ref, u)) - 1) < 1e-10     # the same vector up to a phase
            # it solves the pencil it came from
            r = C[0, :, :, t] @ u - got_l[0, t, n] * (C[0, :, :, t0] @ u)
            assert np.linalg.norm(r) < 1e-10 * np.linalg.norm(C[0, :, :, t0])


def test_optimal_correlator_and_effective_mass_closed_form():
    """Projected with the exact eigenvectors u_n = B^{-1} e_n / |B^{-1} e_n|,
    C_n(t) = lambda_n^t / |B^{-1} e_n|^2 and the effective mass is -log lambda_n
    at every t."""
    lam, B, C = _hermitian_pencil(73)
    nb, nt = len(lam), C.shape[-1]
    _, u = orc.gevp_vectors(C, 1)
    Cn = orc.optimal_correlator(C, u[:, 4])
    Binv = np.linalg.inv(B)
    for n in range(nb):
        expect = lam[n] ** np.arange(nt) / np.linalg.norm(Binv[:, n]) ** 2
        np.testing.assert_allclose(Cn[0, n], expect, rtol=1e-9)
    m = orc.effective_mass(Cn)
    np.testing.assert_allclose(m[0, :, :-1], np.repeat(-np.log(lam)[:, None], nt - 1, axis=1), rtol=1e-9)
    assert np.isnan(m[..., -1]).all()


def test_optimal_correlator_is_phase_invariant_and_diagonalises():
    """The projected correlator does not depend on the eigenvectors' phases,
    and for this pencil the exact eigenvectors make C(t) diagonal."""
    lam, B, C = _hermitian_pencil(79, nb=4)
    _, u = orc.gevp_vectors(C, 1)
    ref = u[:, 3]
    rot = ref * np.exp(1j * np.array([0.3, -1.1, 2.0, 0.7]))[None, :, None]
    np.testing.assert_allclose(orc.optimal_correlator(C, rot), orc.optimal_correlator(C, ref), rtol=1e-12)
    off = ref[0].conj() @ C[0, :, :, 5] @ ref[0].T
    assert np.abs(off - np.diag(np.diag(off))).max() < 1e-10 * np.abs(np.diag(off)).max()


def test_eigenvalue_profiles():
    """g^(b)_i = exp(-(lam_i / sigma_b)^2): one at lam = 0, 1/e at lam = sigma,
    decreasing in lam, unchanged when lam and sigma scale together, and per
    timeslice when lam carries a time axis."""
    lam = np.array([0.0, 0.1, 0.2, 0.4, 1.0])
    g = orc.eigenvalue_profiles(lam, [0.2, 1.0])
    assert g.shape == (2, 5)
    assert g[0, 0] == 1.0 and g[1, 0] == 1.0
    assert abs(g[0, 2] - np.exp(-1.0)) < 1e-15 and abs(g[1, 4] - np.exp(-1.0)) < 1e-15
    assert np.all(np.diff(g, axis=1) < 0)
    np.testing.assert_allclose(orc.eigenvalue_profiles(3 * lam, [0.6, 3.0]), g, rtol=1e-14)  # ratios differ by an ulp
    lam_t = np.stack([lam, 2 * lam])
    gt = orc.eigenvalue_profiles(lam_t, [0.2, 1.0])
    assert gt.shape == (2, 2, 5)
    np.testing.assert_array_equal(gt[0], g)
    np.testing.assert_allclose(gt[1], orc.eigenvalue_profiles(2 * lam, [0.2, 1.0]), rtol=0)
