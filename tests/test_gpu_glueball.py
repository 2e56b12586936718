"""Parity of the A1-+ glueball operators (clover B_i, adjoint covariant
differences, O_1..O_5) against the FP64 oracle, through the C ABI, and
their sign flip under spatial parity and the identity O_5 = -O_4 at full
size.

Tolerance: the path runs in FP64 from the same complex64 links, so the
operators agree to rounding: |dO_n(t)| < 1e-11 of the largest |O_n(t)| of
that timeslice (sums of ~L^3 traces of products of up to six 3 x 3
matrices)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import glueball as og  # noqa: E402
from paper_2609_37723_b300 import synth  # noqa: E402

TOL = 1e-11


@pytest.fixture(scope="module")
def dz():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_37723_b300 import distil
    return distil


def _err(got, ref):
    scale = np.maximum(np.abs(ref).max(axis=-1, keepdims=True), 1e-300)
    return float((np.abs(got - ref) / scale).max())


def _links(L, nt, seed):
    rng = np.random.default_rng(seed)
    return np.stack([synth.haar_su3(rng, (3, L ** 3)) for _ in range(nt)]).astype(np.complex64)


@pytest.mark.parametrize("L,nt", [(4, 3), (5, 2), (3, 1)])
def test_glueball_operators_match_oracle(dz, L, nt):
    U = _links(L, nt, 100 + L)
    O = dz.glueball_operators(torch.from_numpy(U).to("cuda:0"), L).cpu().numpy()
    ref = og.operators(U.astype(np.complex128), L)
    e = _err(O, ref)
    print(f"\nglueball L={L} nt={nt}: {e:.2e}")
    assert e < TOL


def _parity(U, L):
    s = np.arange(L ** 3)
    x, y, z = s % L, (s // L) % L, s // (L * L)
    out = np.empty_like(U)
    for k in range(3):
        d = [int(k == 0), int(k == 1), int(k == 2)]
        src = ((-x - d[0]) % L) + L * (((-y - d[1]) % L) + L * ((-z - d[2]) % L))
        out[:, k] = np.conj(np.swapaxes(U[:, k][:, src], -1, -2))
    return out


def test_glueball_full_size_sampled(dz):
    """The bench workload (L = 24, N_t = 48 links of the meson workload) in
    one call; timeslices 0 and 47 against the oracle, and every timeslice
    against the sign flip under spatial parity."""
    m = synth.meson_config("charm")
    U = m.all_links().astype(np.complex64)
    O = dz.glueball_operators(torch.from_numpy(U).to("cuda:0"), m.L).cpu().numpy()
    ts = [0, m.nt - 1]
    ref = np.stack([og.operators_t(U[t].astype(np.complex128), m.L) for t in ts])
    e = _err(O[ts], ref)
    Op = dz.glueball_operators(torch.from_numpy(np.ascontiguousarray(_parity(U, m.L))).to("cuda:0"),
                               m.L).cpu().numpy()
    ep = _err(Op, -O)
    # summation by parts: O_5 = -O_4 exactly on the periodic lattice
    e45 = float((np.abs(O[:, 3] + O[:, 4]) / np.abs(O).max(axis=-1)).max())
    print(f"\nglueball charm: oracle {e:.2e}, parity {ep:.2e}, O_4 + O_5 {e45:.2e}")
    assert e < TOL
    assert ep < TOL
    assert e45 < TOL
