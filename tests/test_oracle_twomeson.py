"""Pins of the two-meson oracle (oracle/twomeson.py).

The contraction formula is checked against Wick's theorem applied by brute
force: a small engine enumerates every pairing of the quark fields of
<O(t) O(0)^dagger> with the sign of the permutation that brings each pair
together, and evaluates the pairings with einsum over explicit indices.
The same engine fixes the sign convention of the one-meson correlator of
oracle.meson, and the pruning/GEVP weights are checked on a constructed
rank-n matrix whose optimal operators are known."""
import itertools

import numpy as np

from oracle import meson as om
from oracle import twomeson as tm


def _perm_sign(p):
    p = list(p)
    s = 1
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            s = -s
    return s


def wick_terms(fields):
    """fields: list of (flavour, is_bar, label) in product order.  Returns
    [(sign, [(flavour, psi_label, psibar_label), ...])]: every full pairing of
    each flavour's psi with its psi-bar (<psi psi> = <psibar psibar> = 0),
    signed by the permutation that orders the product as
    (psi_1 psibar_s(1))(psi_2 psibar_s(2)) ... flavour by flavour."""
    flavours = sorted({f for f, _, _ in fields})
    per = {}
    for fl in flavours:
        psi = [i for i, (f, b, _) in enumerate(fields) if f == fl and not b]
        bar = [i for i, (f, b, _) in enumerate(fields) if f == fl and b]
        assert len(psi) == len(bar)
        per[fl] = (psi, bar)
    out = []
    for choice in itertools.product(*[list(itertools.permutations(per[fl][1])) for fl in flavours]):
        order, pairs = [], []
        for fl, bars in zip(flavours, choice):
            for i, j in zip(per[fl][0], bars):
                order += [i, j]
                pairs.append((fl, fields[i][2], fields[j][2]))
        out.append((_perm_sign(order), pairs))
    return out


def wick_value(fields, weights, props):
    """sum over indices of prod(weights) x <fields>: weights = [(matrix,
    'xy')], props[flavour] = propagator P with <psi_x psibar_y> = P[x][y]."""
    total = 0j
    for sign, pairs in wick_terms(fields):
        ops = [w for w, _ in weights] + [props[fl] for fl, _, _ in pairs]
        subs = [s for _, s in weights] + [x + y for _, x, y in pairs]
        total += sign * np.einsum(",".join(subs) + "->", *ops)
    return total


def _cg(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def _props(rng, n):
    tau = _cg(rng, (n, n))
    G5 = np.kron(om.GAMMA_5, np.eye(n // 4))
    return tau, G5 @ tau.conj().T @ G5


def test_wick_one_meson_sign():
    """<(ubar M d)(t) (dbar N u)(0)> = -Tr[M S N S~]: the minus of the quark
    loop used by oracle.meson."""
    rng = np.random.default_rng(1)
    n = 4
    S, St = _props(rng, n)
    M, N = _cg(rng, (n, n)), _cg(rng, (n, n))
    fields = [("u", True, "a"), ("d", False, "b"), ("d", True, "e"), ("u", False, "f")]
    got = wick_value(fields, [(M, "ab"), (N, "ef")], {"d": S, "u": St})
    assert abs(got - (-np.trace(M @ S @ N @ St))) < 1e-12 * (1 + abs(got))


def test_wick_matches_meson_correlator():
    """The one-meson correlator of the oracle is the Wick contraction of its
    sink matrix with its source matrix."""
    rng = np.random.default_rng(2)
    nv = 1
    phi_t, phi_0 = _cg(rng, (1, 7, nv, nv)), _cg(rng, (1, 7, nv, nv))
    prof = np.ones((1, nv))
    tau = _cg(rng, (4 * nv, 4 * nv))
    C = om.correlator_t(phi_t, phi_0, tau, prof)
    G5 = np.kron(om.GAMMA_5, np.eye(nv))
    St = G5 @ tau.conj().T @ G5
    fields = [("u", True, "a"), ("d", False, "b"), ("d", True, "e"), ("u", False, "f")]
    for ta in range(3):
        for tb in range(3):
            M = om.sink_matrix(phi_t[0], prof[0], ta)
            N = om.source_matrix(phi_0[0], prof[0], tb)
            got = wick_value(fields, [(M, "ab"), (N, "ef")], {"d": tau, "u": St})
            assert abs(C[0, ta, tb] - got) < 1e-12 * (1 + abs(got))


def test_two_meson_contractions_by_brute_force_wick():
    """<(ubar M1 d)(ubar M2 d)(t) (dbar N2 u)(dbar N1 u)(0)> by brute force
    against the direct-minus-crossed formula of the oracle, on 4 x 4
    spin-mode matrices (N_v = 1) for one momentum pair."""
    rng = np.random.default_rng(3)
    n = 4
    S, St = _props(rng, n)
    M1, M2, N1, N2 = (_cg(rng, (n, n)) for _ in range(4))
    fields = [("u", True, "a"), ("d", False, "b"), ("u", True, "c"), ("d", False, "d"),
              ("d", True, "e"), ("u", False, "f"), ("d", True, "g"), ("u", False, "h")]
    got = wick_value(fields, [(M1, "ab"), (M2, "cd"), (N2, "ef"), (N1, "gh")], {"d": S, "u": St})
    T = lambda M, N: np.trace(M @ S @ N @ St)
    X = lambda A, B, C, D: np.trace(A @ S @ B @ St @ C @ S @ D @ St)
    want = T(M1, N1) * T(M2, N2) + T(M1, N2) * T(M2, N1) - X(M1, N1, M2, N2) - X(M1, N2, M2, N1)
    assert abs(got - want) < 1e-11 * (1 + abs(want))


def test_correlator_sums_the_brute_force_over_back_to_back_pairs():
    """The oracle's momentum-summed correlator equals the brute-force Wick
    value summed over (p, p') with M1 = M(p), M2 = M(-p), N1 = N(p'),
    N2 = N(-p')."""
    rng = np.random.default_rng(4)
    n = 4
    S, St = _props(rng, n)
    keys = [tuple(int(x) for x in p) for p in tm.UNIT_MOMENTA]
    M = {p: _cg(rng, (n, n)) for p in keys}
    N = {p: _cg(rng, (n, n)) for p in keys}
    fields = [("u", True, "a"), ("d", False, "b"), ("u", True, "c"), ("d", False, "d"),
              ("d", True, "e"), ("u", False, "f"), ("d", True, "g"), ("u", False, "h")]
    neg = lambda p: tuple(-x for x in p)
    want = 0j
    for p in keys:
        for q in keys:
            want += wick_value(fields, [(M[p], "ab"), (M[neg(p)], "cd"), (N[neg(q)], "ef"), (N[q], "gh")],
                               {"d": S, "u": St})
    got = tm.correlator_t(M, N, S)
    assert abs(got - want) < 1e-10 * (1 + abs(want))


def test_source_operator_is_the_adjoint():
    """N(p) = gamma_4 M(p, 0)^dagger gamma_4 for the same weights."""
    rng = np.random.default_rng(5)
    nv, nb = 3, 2
    phi = _cg(rng, (7, nv, nv))
    prof = rng.uniform(0.3, 1.0, (nb, nv))
    w = _cg(rng, 3 * nb)
    M = tm.sink_operator(phi, prof, w)
    N = tm.source_operator(phi, prof, w)
    G4 = np.kron(om.GAMMA_4, np.eye(nv))
    assert np.allclose(N, G4 @ M.conj().T @ G4, atol=1e-13)


def test_optimal_weights_recover_the_state_of_a_rank_n_matrix():
    """C(t) = Z diag(lambda^t) Z^dagger of rank 8 in 21 dimensions: the
    optimal operator of the ground state couples to that state only, so
    w^dagger C(t) w decays exactly as lambda_0^t."""
    rng = np.random.default_rng(6)
    nops, n, nt = 21, 8, 6
    Z = _cg(rng, (nops, n))
    lam = np.sort(rng.uniform(0.2, 0.9, n))[::-1]
    C = np.stack([Z @ np.diag(lam ** t) @ Z.conj().T for t in range(nt)], axis=-1)[None]
    w = tm.optimal_weights(C, 1, n, 0, 2)[0]
    corr = np.array([np.vdot(w, C[0, :, :, t] @ w) for t in range(nt)])
    assert np.allclose(corr / corr[0], lam[0] ** np.arange(nt), rtol=1e-8)
    assert abs(np.linalg.norm(w) - 1) < 1e-12
