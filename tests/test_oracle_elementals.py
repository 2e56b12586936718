"""Pins of the oracle's elementals against brute force, closed forms and
invariants (CPU only).

Phi[p,t]_ijk = sum_x exp(-ip.x) eps_abc v_i^a v_j^b v_k^c (Sec. 2.1, the
base elementals that the profiles of the displayed equation rescale).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth

EPS = {p: (1 if sum(1 for a in range(3) for b in range(a + 1, 3) if p[a] > p[b]) % 2 == 0 else -1)
       for p in itertools.permutations(range(3))}


def rand_v(rng, nv, V3):
    return synth.complex_gaussian(rng, (nv, V3, 3))


def brute_elementals(v, L, mom):
    """Literal sum over sites and colour permutations, every ordered (i,j,k).
    The phase is evaluated from the real angle p.x (no modular reduction)."""
    nv, V3, _ = v.shape
    out = np.zeros((len(mom), nv, nv, nv), dtype=np.complex128)
    for q, n in enumerate(mom):
        for s in range(V3):
            x, y, z = s % L, (s // L) % L, s // (L * L)
            ang = 2 * math.pi / L * (n[0] * x + n[1] * y + n[2] * z)
            ph = complex(math.cos(ang), -math.sin(ang))
            for (a, b, c), sgn in EPS.items():
                out[q] += sgn * ph * np.einsum("i,j,k->ijk", v[:, s, a], v[:, s, b], v[:, s, c])
    return out


def packed_from_dense(d, nv):
    i, j, k = orc.triples(nv)
    return d[..., i, j, k]


@pytest.mark.parametrize("L,nv", [(2, 4), (2, 6), (3, 5)])
def test_brute_force(L, nv):
    rng = np.random.default_rng(11 + L * 10 + nv)
    V3 = L ** 3
    v = rand_v(rng, nv, V3)
    mom = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 1], [0, -1, 1]])
    dense = brute_elementals(v, L, mom)
    got = orc.elementals_t(v, L, mom)
    np.testing.assert_allclose(got, packed_from_dense(dense, nv), rtol=0, atol=1e-13)
    # the dense brute force is antisymmetric under every transposition
    np.testing.assert_allclose(dense, -dense.transpose(0, 2, 1, 3), atol=1e-13)
    np.testing.assert_allclose(dense, -dense.transpose(0, 1, 3, 2), atol=1e-13)
    # and unpacking the oracle reproduces all orderings
    np.testing.assert_allclose(orc.unpack(got, nv), dense, atol=1e-13)


def test_single_site_is_determinant():
    rng = np.random.default_rng(5)
    v = rand_v(rng, 3, 1)
    got = orc.elementals_t(v, 1, np.array([[0, 0, 0]]))
    det = np.linalg.det(np.stack([v[0, 0], v[1, 0], v[2, 0]], axis=1))
    assert got.shape == (1, 1)
    assert abs(got[0, 0] - det) < 1e-14


def test_plane_wave_closed_form():
    """v_i(x) = exp(i q_i.x) e_{c_i} / sqrt(V3) gives
    Phi_ijk(p) = eps_{c_i c_j c_k} V3^{-1/2} delta(p = q_i + q_j + q_k mod L)."""
    L, V3 = 4, 64
    rng = np.random.default_rng(3)
    nv = 7
    qs = rng.integers(-2, 3, size=(nv, 3))
    cs = rng.integers(0, 3, size=nv)
    cs[:3] = [0, 1, 2]
    cs[3:6] = [2, 0, 1]
    xyz = orc.site_coords(L)
    v = np.zeros((nv, V3, 3), dtype=np.complex128)
    for i in range(nv):
        v[i, :, cs[i]] = np.exp(2j * np.pi / L * (xyz @ qs[i])) / math.sqrt(V3)
    # momenta that hit some triples with distinct colours, plus unrelated ones
    mom = np.array([qs[0] + qs[1] + qs[2], qs[3] + qs[4] + qs[5], qs[0] + qs[4] + qs[5],
                    [0, 0, 0], [1, 0, 0], [-1, 2, 1]]) % L
    got = orc.elementals_t(v, L, mom)
    i_, j_, k_ = orc.triples(nv)
    expect = np.zeros_like(got)
    for r, (i, j, k) in enumerate(zip(i_, j_, k_)):
        cperm = (cs[i], cs[j], cs[k])
        if len(set(cperm)) < 3:
            continue
        for q, n in enumerate(mom):
            if np.all((qs[i] + qs[j] + qs[k] - n) % L == 0):
                expect[q, r] = EPS[cperm] / math.sqrt(V3)
    np.testing.assert_allclose(got, expect, atol=1e-14)
    assert np.count_nonzero(np.abs(expect) > 0) >= 3


def _oracle(v, L, mom):
    return orc.elementals_t(v, L, mom)


def test_mode_reversal_antisymmetry():
    rng = np.random.default_rng(7)
    L, nv = 3, 6
    v = rand_v(rng, nv, L ** 3)
    mom = np.array([[0, 0, 0], [1, 1, 0]])
    a = _oracle(v, L, mom)
    b = _oracle(v[::-1].copy(), L, mom)
    # (i,j,k) of the reversed set is (n-1-k, n-1-j, n-1-i) of the original:
    # an odd permutation of the three slots.
    for r, (i, j, k) in enumerate(zip(*orc.triples(nv))):
        rr = orc.triple_rank(nv - 1 - k, nv - 1 - j, nv - 1 - i)
        np.testing.assert_allclose(b[:, r], -a[:, rr], atol=1e-14)


def random_su3(rng):
    z = synth.complex_gaussian(rng, (3, 3))
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return q / np.linalg.det(q) ** (1.0 / 3.0)


def test_su3_gauge_invariance():
    rng = np.random.default_rng(9)
    L, nv = 3, 5
    V3 = L ** 3
    v = rand_v(rng, nv, V3)
    U = np.stack([random_su3(rng) for _ in range(V3)])
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)
    vr = np.einsum("xab,ixb->ixa", U, v)
    mom = np.array([[0, 0, 0], [1, 0, 0], [1, 2, 0]])
    np.testing.assert_allclose(_oracle(vr, L, mom), _oracle(v, L, mom), atol=1e-13)


def test_translation_gives_phase():
    rng = np.random.default_rng(13)
    L, nv = 4, 5
    V3 = L ** 3
    v = rand_v(rng, nv, V3)
    shift = np.array([1, 2, 3])
    xyz = orc.site_coords(L)
    src = (xyz + shift) % L
    idx = src[:, 0] + L * (src[:, 1] + L * src[:, 2])
    vs = v[:, idx, :]                                  # v'(x) = v(x + s)
    mom = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1], [1, 1, 1]])
    a = _oracle(v, L, mom)
    b = _oracle(vs, L, mom)
    ph = np.exp(2j * np.pi / L * (mom @ shift))        # exp(i p.s)
    np.testing.assert_allclose(b, a * ph[:, None], atol=1e-13)


def test_vector_phases():
    rng = np.random.default_rng(17)
    L, nv = 2, 6
    v = rand_v(rng, nv, L ** 3)
    th = rng.uniform(0, 2 * np.pi, size=nv)
    mom = np.array([[0, 0, 0], [1, 1, 0]])
    a = _oracle(v, L, mom)
    b = _oracle(v * np.exp(1j * th)[:, None, None], L, mom)
    i, j, k = orc.triples(nv)
    np.testing.assert_allclose(b, a * np.exp(1j * (th[i] + th[j] + th[k]))[None], atol=1e-13)


def test_real_fields_conjugate_momentum():
    rng = np.random.default_rng(19)
    L, nv = 3, 5
    v = rng.standard_normal((nv, L ** 3, 3)).astype(np.complex128)
    mom = np.array([[1, 0, 0], [-1, 0, 0], [1, 2, 0], [-1, -2, 0]])
    a = _oracle(v, L, mom)
    np.testing.assert_allclose(a[1], np.conj(a[0]), atol=1e-13)
    np.testing.assert_allclose(a[3], np.conj(a[2]), atol=1e-13)


def test_generated_workload_shapes():
    p = synth.config(1)
    v = p.eigvecs(0)
    assert v.shape == (16, 512, 3) and v.dtype == np.complex128
    m = v.reshape(16, -1)
    np.testing.assert_allclose(m.conj() @ m.T, np.eye(16), atol=1e-13)
    assert p.perambulator(2).shape == (64, 64)
    assert orc.n_triples(16) == 560
