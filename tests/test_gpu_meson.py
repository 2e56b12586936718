"""Parity of the meson path (elementals with covariant displacements, the
profiled 21 x 21 correlation matrix, SVD pruning and the pruned GEVP)
against the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances: the elementals per (t, p, d) relative to their largest entry,
5e-8 (the FP16X6 elementals scheme keeps 29 to 30 bits of every operand
row once its 2-norm is capped for exact coherent sums, and a row's largest
entry is a few times its typical one); the correlation matrix per entry relative to the magnitude of the
two operators it couples (sqrt of their largest row/column entries), 1e-6
-- the entries of the 21 x 21 matrix span five orders of magnitude, so a
plain per-entry gate would demand 1e-11 of the matrix on its smallest
entries -- and relative to the largest entry of C(p, t), 3e-7 (the rows that can
sum coherently are split with a capped norm so that the tensor core's
leading-slice sums stay exact, which leaves them 29 to 30 bits); pruning in
FP64 to 1e-10 of the matrix scale; the eigenvalues of the pruned GEVP to
1e-5 relative (the GEVP amplifies the correlator's errors by the
conditioning of C(t0)).  The plain per-entry errors are printed."""
import numpy as np
import pytest

from parity import max_c_error, max_c_operator_scaled_error, max_c_scaled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import meson as om  # noqa: E402
from paper_2609_37723_b300 import synth  # noqa: E402

TOL_PHI = 5e-8
TOL_C = 1e-6        # relative to the operators' magnitude
TOL_C_SCALED = 3e-7  # relative to the largest entry of C(p, t)


@pytest.fixture(scope="module")
def dz():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_37723_b300 import distil
    return distil


def _phi_err(got, ref):
    scale = np.maximum(np.abs(ref).max(axis=(-2, -1), keepdims=True), 1e-300)
    return float((np.abs(got - ref) / scale).max())


def _ragged():
    sig = [0.2, 0.5, 1.1]
    base = synth.Problem("L5_Nt3_Nv13_meson", 5, 3, 13, np.array([[0, 0, 0]], dtype=np.int32),
                         synth.gaussian_profiles(13, sig), 0.5, np.dtype(np.complex64), 9, 0)
    return synth.MesonProblem(base, 5, 1)


def _inputs(m, ts=None):
    v = m.all_eigvecs(ts)
    U = m.all_links(ts)
    tau = m.all_perambulators(ts)
    return v, U, tau


def _gpu_chain(dz, m, v, U, tau):
    dev = torch.device("cuda:0")
    vd = torch.from_numpy(np.ascontiguousarray(v.astype(np.complex64))).to(dev)
    Ud = torch.from_numpy(np.ascontiguousarray(U.astype(np.complex64))).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(tau.astype(np.complex64))).to(dev)
    pd = torch.from_numpy(np.ascontiguousarray(m.prof)).to(dev)
    phi = dz.meson_elementals(vd, Ud, m.L, m.mom)
    C = dz.meson_correlate(phi, phi[0].contiguous(), td, pd)
    torch.cuda.synchronize()
    return phi, C


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_meson_elementals_and_correlator(dz, which):
    m = synth.meson_config("small") if which == "small" else _ragged()
    v, U, tau = _inputs(m)
    phi, C = _gpu_chain(dz, m, v, U, tau)
    ref_phi = om.elementals(v.astype(np.complex128), U.astype(np.complex128), m.L, m.mom)
    e_phi = _phi_err(phi.cpu().numpy(), ref_phi)
    ref_C = om.correlator(ref_phi, ref_phi[0], tau.astype(np.complex128), m.prof)
    got = C.cpu().numpy()
    e_C, e_s = max_c_operator_scaled_error(got, ref_C), max_c_scaled_error(got, ref_C)
    print(f"\n{m.name}: elementals {e_phi:.2e}, C operator-scaled {e_C:.2e}, matrix-scaled {e_s:.2e}, "
          f"per entry {max_c_error(got, ref_C):.2e}")
    assert e_phi < TOL_PHI
    assert e_C < TOL_C and e_s < TOL_C_SCALED


def _eig_match_err(got, ref):
    """Largest relative error of the eigenvalues of every (p, t) matched as
    multisets (each reference eigenvalue takes the nearest unmatched one:
    complex-conjugate pairs share a modulus, so the sorted orders can differ)."""
    worst = 0.0
    for idx in np.ndindex(ref.shape[:-1]):
        left = list(got[idx])
        for r in sorted(ref[idx], key=lambda z: -abs(z)):
            k = int(np.argmin([abs(g - r) for g in left]))
            worst = max(worst, abs(left[k] - r) / max(abs(r), 1e-300))
            left.pop(k)
    return worst


def _phase_fix(u):
    out = u.copy()
    for q in range(u.shape[0]):
        for m in range(u.shape[2]):
            col = out[q, :, m]
            k = int(np.argmax(np.abs(col)))
            out[q, :, m] = col * (np.conj(col[k]) / abs(col[k]))
    return out


def test_meson_prune_matches_oracle(dz):
    rng = np.random.default_rng(3)
    for nops, nkeep in [(21, 8), (30, 16), (5, 5)]:
        C = (rng.standard_normal((2, nops, nops, 4)) + 1j * rng.standard_normal((2, nops, nops, 4)))
        Ct, Un, sv = dz.meson_prune(torch.from_numpy(C).to("cuda:0"), 1, nkeep)
        rCt, rUn, rsv = om.prune(C, 1, nkeep)
        rUn = _phase_fix(rUn)
        # Ct of the phase-fixed basis
        rCt = np.einsum("qam,qabt,qbn->qmnt", rUn.conj(), C, rUn)
        scale = np.abs(C).max()
        assert np.abs(sv.cpu().numpy() - rsv).max() < 1e-10 * rsv.max()
        assert np.abs(Un.cpu().numpy() - rUn).max() < 1e-9
        assert np.abs(Ct.cpu().numpy() - rCt).max() < 1e-10 * scale


def test_meson_chain_pruned_gevp(dz):
    m = synth.meson_config("small")
    v, U, tau = _inputs(m)
    phi, C = _gpu_chain(dz, m, v, U, tau)
    Ct, Un, sv = dz.meson_prune(C, m.t_prune, m.nkeep)
    lam = dz.gevp(Ct, 0).cpu().numpy()
    ref_phi = om.elementals(v.astype(np.complex128), U.astype(np.complex128), m.L, m.mom)
    ref_C = om.correlator(ref_phi, ref_phi[0], tau.astype(np.complex128), m.prof)
    rCt, rUn, rsv = om.prune(ref_C, m.t_prune, m.nkeep)
    ref_lam = om.gevp(rCt, 0)
    assert np.abs(sv.cpu().numpy() - rsv).max() < 1e-6 * rsv.max()
    # the projector onto the kept singular vectors is basis-free
    P = np.einsum("qam,qbm->qab", Un.cpu().numpy(), Un.cpu().numpy().conj())
    rP = np.einsum("qam,qbm->qab", rUn, rUn.conj())
    assert np.abs(P - rP).max() < 1e-5
    err = _eig_match_err(lam[:, 1:], ref_lam[:, 1:])
    print(f"\npruned GEVP max rel err {err:.2e}")
    assert err < 1e-5


def test_meson_full_size_sampled(dz):
    """The bench workload (L = 24, N_t = 48, N_v = 200) in the bench's launch
    configuration (all timeslices in one call); timeslices 0 (the source)
    and 47 against the oracle."""
    m = synth.meson_config("charm")
    v, U, tau = _inputs(m)
    phi, C = _gpu_chain(dz, m, v, U, tau)
    ts = [0, m.nt - 1]
    ref_phi = np.stack([om.elementals_t(v[t].astype(np.complex128), U[t].astype(np.complex128), m.L, m.mom)
                        for t in ts])
    got_phi = phi[ts].cpu().numpy()
    e_phi = _phi_err(got_phi, ref_phi)
    ref_C = om.correlator(ref_phi, ref_phi[0], tau[ts].astype(np.complex128), m.prof)
    got_C = C[..., ts].cpu().numpy()
    e_C, e_s = max_c_operator_scaled_error(got_C, ref_C), max_c_scaled_error(got_C, ref_C)
    print(f"\ncharm sampled: elementals {e_phi:.2e}, C operator-scaled {e_C:.2e}, matrix-scaled {e_s:.2e}, "
          f"per entry {max_c_error(got_C, ref_C):.2e}")
    assert e_phi < TOL_PHI
    assert e_C < TOL_C and e_s < TOL_C_SCALED
    assert np.all(np.isfinite(C.cpu().numpy()))


def test_meson_rejects_other_modes(dz):
    m = synth.meson_config("small")
    dev = torch.device("cuda:0")
    v = torch.zeros((1, m.nv, m.V3, 3), dtype=torch.complex64, device=dev)
    U = torch.zeros((1, 3, m.V3, 3, 3), dtype=torch.complex64, device=dev)
    with pytest.raises(dz.DistilError) as e:
        dz.meson_elementals(v, U, m.L, m.mom, mode="fp64", workspace=torch.empty(256, dtype=torch.uint8,
                                                                                  device=dev))
    assert e.value.status == 5
