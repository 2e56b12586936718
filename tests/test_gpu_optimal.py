"""GEVP eigenvectors, optimal-operator correlators and the one-timeslice
correlator entry point on the GPU, against the FP64 oracle.

Sec. 2.1: the N_B x N_B correlation matrix of the profiled elementals feeds
a GEVP; its eigenvectors weight the profiled operators into the optimal
operator of each state, whose correlator gives the effective masses.
Eigenvectors are unique up to a phase: they are compared through
|<u_gpu, u_oracle>| and through the phase-independent projected
correlators."""
import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth
from parity import max_c_error

pytestmark = pytest.mark.gpu


def T(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def pencil(seed, nb=6, nt=10):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(0.2, 0.95, nb))[::-1]
    B = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
    A = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
    C = np.zeros((2, nb, nb, nt), dtype=np.complex128)
    for t in range(nt):
        C[0, :, :, t] = B.conj().T @ np.diag(lam ** t) @ B         # Hermitian pencil
        C[1, :, :, t] = A @ np.diag(lam ** t) @ B                  # general pencil
    return C


@pytest.fixture(scope="module")
def c1_C():
    p = synth.config(1)
    v = p.all_eigvecs()
    tau = p.all_perambulators()
    phi = orc.elementals(v, p.L, p.mom)
    return orc.correlator(phi, phi[0], tau, p.prof)


@pytest.mark.parametrize("which", ["pencil", "c1"])
def test_gevp_vectors_match_oracle(cuda_lib, c1_C, which):
    from paper_2609_37723_b300 import distil
    C = pencil(5) if which == "pencil" else c1_C
    t0 = 2
    lam_ref, u_ref = orc.gevp_vectors(C, t0)
    lam, vecs = distil.gevp_range(T(C), t0, want_vectors=True)
    lam, vecs = lam.cpu().numpy(), vecs.cpu().numpy()
    npm, nb, _, nt = C.shape
    for q in range(npm):
        for t in range(nt):
            if t == t0:
                continue            # lambda = 1 (all degenerate): any basis is an eigenbasis
            np.testing.assert_allclose(lam[q, t], lam_ref[q, t], rtol=1e-10, atol=1e-14 * np.abs(lam_ref[q, t]).max())
            for n in range(nb):
                u = vecs[q, t, n]
                assert abs(np.linalg.norm(u) - 1) < 1e-12
                k = np.argmax(np.abs(u))
                assert abs(u[k].imag) <= 1e-15 * abs(u[k]) and u[k].real > 0
                overlap = abs(np.vdot(u_ref[q, t, n], u))
                assert overlap > 1 - 1e-10, (q, t, n, overlap)
                # and it solves the pencil
                r = C[q, :, :, t] @ u - lam[q, t, n] * (C[q, :, :, t0] @ u)
                assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(C[q, :, :, t])


def test_gevp_range_touches_only_its_timeslices(cuda_lib):
    import torch
    from paper_2609_37723_b300 import distil
    C = pencil(9)
    npm, nb, _, nt = C.shape
    lam = torch.full((npm, nt, nb), complex(5.0, 5.0), dtype=torch.complex128, device="cuda")
    vecs = torch.full((npm, nt, nb, nb), complex(5.0, 5.0), dtype=torch.complex128, device="cuda")
    distil.gevp_range(T(C), 1, t_begin=4, t_count=3, lam=lam, vecs=vecs)
    full = distil.gevp(T(C), 1).cpu().numpy()
    got = lam.cpu().numpy()
    assert np.array_equal(got[:, 4:7], full[:, 4:7])
    assert np.all(got[:, :4] == 5 + 5j) and np.all(got[:, 7:] == 5 + 5j)
    assert np.all(vecs.cpu().numpy()[:, :4] == 5 + 5j)


def test_optimal_correlator_and_effective_mass(cuda_lib, c1_C):
    """Projected correlators and effective masses from the GPU eigenvectors
    against the oracle's projection with its own eigenvectors (the
    projection does not depend on the eigenvectors' phases)."""
    from paper_2609_37723_b300 import distil
    for C, t0, td in ((pencil(13), 1, 4), (c1_C, 2, 4)):
        _, u_ref = orc.gevp_vectors(C, t0)
        ref = orc.optimal_correlator(C, u_ref[:, td])
        m_ref = orc.effective_mass(ref)
        _, vecs = distil.gevp_range(T(C), t0, want_vectors=True)
        copt, meff = distil.optimal(T(C), vecs, td)
        copt, meff = copt.cpu().numpy(), meff.cpu().numpy()
        scale = np.abs(ref).max(axis=-1, keepdims=True)
        assert (np.abs(copt - ref) / scale).max() < 1e-10
        fin = np.isfinite(m_ref)
        assert np.array_equal(fin, np.isfinite(meff))
        assert np.abs(meff[fin] - m_ref[fin]).max() < 1e-8
    # the Hermitian pencil's ground state has the exact effective mass -log lambda_0
    rng = np.random.default_rng(13)
    lam0 = np.sort(rng.uniform(0.2, 0.95, 6))[::-1][0]
    copt, meff = distil.optimal(T(pencil(13)), distil.gevp_range(T(pencil(13)), 1, want_vectors=True)[1], 4)
    assert np.abs(meff.cpu().numpy()[0, 0, :-1] + np.log(lam0)).max() < 1e-9


@pytest.mark.parametrize("mode", ["fp64", "fp16x6"])
def test_correlate_slice_matches_full_call(cuda_lib, mode):
    """One timeslice at a time into column t of C gives the matrix of the
    whole-range call (the tensor-core path bit for bit: its normalisation and
    reductions are per timeslice and deterministic)."""
    import torch
    from paper_2609_37723_b300 import distil
    p = synth.small(4, 3, 12, mom=[(0, 0, 0), (1, 0, 0)], sigmas=(0.4, 0.9, 1.3), seed_cfg=17)
    cdt = np.complex128 if mode == "fp64" else np.complex64
    v = p.all_eigvecs().astype(cdt)
    tau = T(p.all_perambulators().astype(cdt))
    phi = distil.elementals(T(v), p.L, p.mom, mode)
    prof = T(p.prof)
    full = distil.correlate(phi, phi[0].contiguous(), tau, prof, mode).cpu().numpy()
    C = torch.full((p.np_, p.nb, p.nb, p.nt), complex(3.0, 3.0), dtype=torch.complex128, device="cuda")
    for t in (2, 0):
        distil.correlate_slice(phi[t].contiguous(), phi[0].contiguous(), tau[t].contiguous(), prof, prof, C, t,
                               mode)
    got = C.cpu().numpy()
    assert np.all(got[..., 1] == 3 + 3j)              # untouched column
    for t in (0, 2):
        if mode == "fp64":
            assert max_c_error(got[..., t:t + 1], full[..., t:t + 1]) < 1e-13
        else:
            assert np.array_equal(got[..., t], full[..., t])


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("fp16x6", 1e-6)])
def test_per_timeslice_profiles_every_mode(cuda_lib, mode, tol):
    """Profiles g^(a)[t] (Sec. 2.1) in the plain and the tensor-core paths:
    the whole-range call with per-t profiles and the one-timeslice call with
    separate sink (g[t]) and source (g[0]) profiles, against the oracle."""
    import torch
    from paper_2609_37723_b300 import distil
    rng = np.random.default_rng(21)
    p = synth.small(3, 3, 10, mom=[(0, 0, 0), (0, 1, 1)], sigmas=(0.5, 1.0), seed_cfg=23)
    cdt = np.complex128 if mode == "fp64" else np.complex64
    v = p.all_eigvecs().astype(cdt)
    tau_h = p.all_perambulators().astype(cdt)
    prof_t = rng.uniform(0.1, 1.0, size=(p.nt, 2, p.nv))
    phi_ref = orc.elementals(v, p.L, p.mom)
    ref = orc.correlator(phi_ref, phi_ref[0], tau_h, prof_t, prof_per_t=True)
    phi = T(phi_ref.astype(np.complex128 if mode != "fp32" else np.complex64))
    tau = T(tau_h)
    got = distil.correlate(phi, phi[0].contiguous(), tau, T(prof_t), mode, prof_per_t=True).cpu().numpy()
    assert max_c_error(got, ref) < tol
    C = torch.zeros((p.np_, 2, 2, p.nt), dtype=torch.complex128, device="cuda")
    for t in range(p.nt):
        distil.correlate_slice(phi[t].contiguous(), phi[0].contiguous(), tau[t].contiguous(), T(prof_t[t]),
                               T(prof_t[0]), C, t, mode)
    assert max_c_error(C.cpu().numpy(), ref) < tol


def test_eigenvalue_profiles_match_oracle(cuda_lib):
    """Profiles from the Laplacian eigenvalues (Sec. 2.1) on the GPU against
    the oracle's exp(-(lam/sigma)^2), per timeslice."""
    from paper_2609_37723_b300 import distil
    p = synth.config(2)
    lam = np.stack([p.laplacian_eigenvalues(t) for t in range(4)])
    sig = [0.1, 0.3, 0.6, 1.2]
    got = distil.profiles_eigen(T(lam), sig).cpu().numpy()
    ref = orc.eigenvalue_profiles(lam, sig)
    assert got.shape == (4, 4, p.nv)
    assert np.abs(got - ref).max() < 1e-15
    one = distil.profiles_eigen(T(lam[0]), sig).cpu().numpy()
    assert np.array_equal(one, got[0])


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("fp16x6", 1e-6)])
def test_correlator_with_eigenvalue_profiles(cuda_lib, mode, tol):
    """The chain with per-timeslice eigenvalue profiles made on the GPU:
    elementals -> C_ab(t) (sink g[t], source g[0]) against the oracle."""
    from paper_2609_37723_b300 import distil
    p = synth.small(4, 3, 14, mom=[(0, 0, 0), (1, 0, 1)], sigmas=(0.5,), seed_cfg=41,
                    dtype=np.complex128 if mode == "fp64" else np.complex64)
    lam = np.stack([p.laplacian_eigenvalues(t) for t in range(p.nt)])
    sig = [0.08, 0.15, 0.4]
    v, tau = p.all_eigvecs(), p.all_perambulators()
    prof_ref = orc.eigenvalue_profiles(lam, sig)
    phi_ref = orc.elementals(v, p.L, p.mom)
    ref = orc.correlator(phi_ref, phi_ref[0], tau, prof_ref, prof_per_t=True)
    prof = distil.profiles_eigen(T(lam), sig)
    phi = distil.elementals(T(v), p.L, p.mom, mode)
    got = distil.correlate(phi, phi[0].contiguous(), T(tau), prof, mode, prof_per_t=True).cpu().numpy()
    print(f"eigenvalue profiles {mode}: strict per-entry {max_c_error(got, ref):.2e}")
    assert max_c_error(got, ref) < tol
