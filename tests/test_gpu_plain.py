"""Parity of the plain FP64 / FP32 CUDA paths with the FP64 oracle, through
the C ABI.  Tolerances: FP64 1e-12 per C_ab(t) entry and per elemental
(relative to the largest |Phi| of its (t, p)); FP32 from its arithmetic:
FP32 sums over K terms carry ~u*sqrt(K) relative error, u = 2^-24, with
K = 3 V3 <= 1e5 for the elementals -> gate 1e-4 on elementals and C."""
import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth
from parity import max_c_error, normwise, phi_error

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4


def T(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def c1():
    p = synth.config(1)
    v = p.all_eigvecs()
    tau = p.all_perambulators()
    phi = orc.elementals(v, p.L, p.mom)
    C = orc.correlator(phi, phi[0], tau, p.prof)
    return p, v, tau, phi, C


def test_elementals_fp64_c1(cuda_lib, c1):
    from paper_2609_37723_b300 import distil
    p, v, tau, phi, C = c1
    got = distil.elementals(T(v), p.L, p.mom, "fp64").cpu().numpy()
    assert got.shape == phi.shape
    assert phi_error(got, phi) < TOL64


def test_correlate_fp64_c1(cuda_lib, c1):
    from paper_2609_37723_b300 import distil
    p, v, tau, phi, C = c1
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), "fp64").cpu().numpy()
    assert max_c_error(got, C) < TOL64


def test_chain_fp64_c1(cuda_lib, c1):
    """GPU elementals feeding the GPU correlator, against the oracle chain."""
    from paper_2609_37723_b300 import distil
    p, v, tau, phi, C = c1
    ph = distil.elementals(T(v), p.L, p.mom, "fp64")
    got = distil.correlate(ph, ph[0].contiguous(), T(tau), T(p.prof), "fp64").cpu().numpy()
    assert max_c_error(got, C) < TOL64


def test_fp32_c1(cuda_lib, c1):
    from paper_2609_37723_b300 import distil
    p, v, tau, phi, C = c1
    v32, tau32 = v.astype(np.complex64), tau.astype(np.complex64)
    ref_phi = orc.elementals(v32, p.L, p.mom)
    ref_C = orc.correlator(ref_phi, ref_phi[0], tau32, p.prof)
    ph = distil.elementals(T(v32), p.L, p.mom, "fp32")
    assert phi_error(ph.cpu().numpy(), ref_phi) < TOL32
    got = distil.correlate(ph, ph[0].contiguous(), T(tau32), T(p.prof), "fp32").cpu().numpy()
    assert max_c_error(got, ref_C) < TOL32


@pytest.mark.parametrize("L,nt,nv,mom,nb", [
    (3, 2, 5, [(0, 0, 0)], 1),
    (3, 1, 7, [(1, 0, 0), (0, -1, 2), (1, 1, 1)], 2),
    (2, 3, 17, [(0, 0, 0), (1, 1, 0)], 3),
    (1, 2, 3, [(0, 0, 0)], 2),
    (4, 2, 66, [(1, 0, 0)], 2),      # ragged 64-wide tiles in every GEMM dimension
])
def test_odd_shapes_fp64(cuda_lib, L, nt, nv, mom, nb):
    from paper_2609_37723_b300 import distil
    p = synth.small(L, nt, nv, mom=mom, sigmas=[0.3, 0.7, 1.4][:nb], seed_cfg=nv)
    v = p.all_eigvecs()
    tau = p.all_perambulators()
    phi = orc.elementals(v, p.L, p.mom)
    got_phi = distil.elementals(T(v), p.L, p.mom, "fp64").cpu().numpy()
    assert phi_error(got_phi, phi) < TOL64
    ts = [0, nt - 1] if nv > 20 else None
    C = orc.correlator(phi, phi[0], tau, p.prof, ts=ts)
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), "fp64").cpu().numpy()
    sel = slice(None) if ts is None else ts
    assert max_c_error(got[..., sel], C[..., sel]) < TOL64


@pytest.mark.parametrize("nv", [1, 2])
def test_fewer_than_three_modes(cuda_lib, nv):
    """No triple i<j<k exists: the elementals are empty and C vanishes."""
    import torch
    from paper_2609_37723_b300 import distil
    p = synth.small(2, 2, nv, sigmas=[0.5])
    v = p.all_eigvecs()
    ph = distil.elementals(T(v), p.L, p.mom, "fp64")
    assert ph.shape[-1] == 0
    tau = p.all_perambulators()
    C = distil.correlate(ph, ph[0].contiguous(), T(tau), T(p.prof), "fp64").cpu().numpy()
    assert np.all(C == 0)


def test_profiles_per_timeslice(cuda_lib):
    from paper_2609_37723_b300 import distil
    rng = np.random.default_rng(3)
    p = synth.small(2, 3, 6, sigmas=[0.4, 0.9])
    v = p.all_eigvecs()
    tau = p.all_perambulators()
    phi = orc.elementals(v, p.L, p.mom)
    prof_t = rng.uniform(0.1, 1.0, size=(p.nt, 2, p.nv))
    C = orc.correlator(phi, phi[0], tau, prof_t, prof_per_t=True)
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(prof_t), "fp64", prof_per_t=True).cpu().numpy()
    assert max_c_error(got, C) < TOL64


def test_c2_sampled_timeslices(cuda_lib):
    """Workload 2 (L=24, N_v=64, 3 momenta, 4 profiles) on four timeslices,
    every momentum, FP64 and FP32 GPU paths against the oracle."""
    from paper_2609_37723_b300 import distil
    p = synth.config(2)
    ts = [0, 1, 24, 47]
    v = p.all_eigvecs(ts)
    tau = p.all_perambulators(ts)
    ref_phi = orc.elementals(v, p.L, p.mom)
    ref_C = orc.correlator(ref_phi, ref_phi[0], tau, p.prof)
    v64, tau64 = v.astype(np.complex128), tau.astype(np.complex128)
    ph = distil.elementals(T(v64), p.L, p.mom, "fp64")
    assert phi_error(ph.cpu().numpy(), ref_phi) < TOL64
    got = distil.correlate(ph, ph[0].contiguous(), T(tau64), T(p.prof), "fp64").cpu().numpy()
    assert max_c_error(got, ref_C) < TOL64
    ph32 = distil.elementals(T(v), p.L, p.mom, "fp32")
    assert phi_error(ph32.cpu().numpy(), ref_phi) < TOL32
    got32 = distil.correlate(ph32, ph32[0].contiguous(), T(tau), T(p.prof), "fp32").cpu().numpy()
    print(f"c2 fp32: strict per-entry {max_c_error(got32, ref_C):.2e}, normwise {normwise(got32, ref_C):.2e}")
    assert max_c_error(got32, ref_C) < TOL32


# ------------------------------------------------------------------ GEVP

def test_gevp_constructed(cuda_lib):
    from paper_2609_37723_b300 import distil
    rng = np.random.default_rng(5)
    nb, nt, t0 = 6, 10, 2
    C = np.zeros((3, nb, nb, nt), dtype=np.complex128)
    lams = []
    for q in range(3):
        lam = np.sort(rng.uniform(0.1, 0.95, nb))[::-1]
        A = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
        B = synth.complex_gaussian(rng, (nb, nb)) + 3 * np.eye(nb)
        for t in range(nt):
            C[q, :, :, t] = A @ np.diag(lam ** t) @ (B if q < 2 else A.conj().T)
        lams.append(lam)
    got = distil.gevp(T(C), t0).cpu().numpy()
    # eigenvalue perturbation bounds are normwise (Bauer-Fike): a small
    # eigenvalue carries an absolute error of order eps times the largest one
    for q in range(3):
        for t in range(nt):
            expect = lams[q] ** (t - t0)
            scale = np.abs(expect).max()
            np.testing.assert_allclose(got[q, t], expect[np.argsort(-np.abs(expect))], rtol=1e-9,
                                       atol=1e-12 * scale)
            np.testing.assert_allclose(got[q, t], orc.gevp(C, t0)[q, t], rtol=1e-9, atol=1e-12 * scale)


def test_gevp_of_c1(cuda_lib, c1):
    from paper_2609_37723_b300 import distil
    p, v, tau, phi, C = c1
    ref = orc.gevp(C, 2)
    got = distil.gevp(T(C), 2).cpu().numpy()
    # conditioning of C(t0) bounds the attainable accuracy; the matrices here
    # are small and well separated
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-12 * np.abs(ref).max())


def test_gevp_singular_gives_nan(cuda_lib):
    from paper_2609_37723_b300 import distil
    C = np.zeros((1, 3, 3, 4), dtype=np.complex128)
    C[0, :, :, 1] = np.eye(3)
    got = distil.gevp(T(C), 0).cpu().numpy()
    assert np.all(np.isnan(got))
