"""The seeded synthetic inputs follow the stated recipe: shapes and dtypes of
each workload, orthonormal eigenvectors, perambulator decay, profile and
momentum sets, and reproducible, independent random streams."""
import numpy as np
import pytest

from paper_2609_37723_b300 import synth


@pytest.mark.parametrize("cid,L,nt,nv,np_,nb,dtype", [
    (1, 8, 8, 16, 2, 3, np.complex128),
    (2, 24, 48, 64, 3, 4, np.complex64),
    (3, 32, 64, 128, 5, 6, np.complex64),
    (5, 48, 96, 256, 9, 8, np.complex64),
])
def test_workload_parameters(cid, L, nt, nv, np_, nb, dtype):
    p = synth.config(cid)
    assert (p.L, p.nt, p.nv, p.np_, p.nb) == (L, nt, nv, np_, nb)
    assert np.dtype(p.dtype) == np.dtype(dtype)
    assert (p.mom[0] == 0).all()                     # zero momentum first
    assert p.prof.shape == (nb, nv) and (p.prof[:, 0] == 1.0).all()   # 0-based: g_0 = 1


def test_profiles_and_sigmas():
    p3 = synth.config(3)
    i = np.arange(128) / 128
    for a in range(6):
        sig = 0.2 * 6.0 ** (a / 5)
        np.testing.assert_allclose(p3.prof[a], np.exp(-i ** 2 / sig ** 2), rtol=1e-15)
    p2 = synth.config(2)
    np.testing.assert_allclose(p2.prof[3], 1 - np.arange(64) / 64)   # the index-linear profile
    np.testing.assert_allclose(p2.prof[:3], synth.gaussian_profiles(64, [0.3, 0.6, 1.0]))


def test_workload4_ensemble_nv_draws():
    nvs = [synth.config(4, c).nv for c in range(16)]
    assert set(nvs) <= {64, 96, 128} and len(set(nvs)) > 1
    assert nvs == [synth.config(4, c).nv for c in range(16)]     # seeded, reproducible
    assert synth.config(4, 0).mom.shape == (7, 3)


def test_eigenvectors_orthonormal_and_reproducible():
    p = synth.small(3, 3, 10, seed_cfg=4)
    for t in range(3):
        m = p.eigvecs(t).reshape(10, -1)
        np.testing.assert_allclose(m.conj() @ m.T, np.eye(10), atol=1e-13)
    assert np.array_equal(p.eigvecs(1), synth.small(3, 3, 10, seed_cfg=4).eigvecs(1))
    assert not np.allclose(p.eigvecs(1), p.eigvecs(2))          # timeslices draw independently
    assert not np.allclose(p.eigvecs(1), synth.small(3, 3, 10, seed_cfg=5).eigvecs(1))


def test_perambulator_statistics_and_decay():
    p = synth.small(2, 6, 64, seed_cfg=1, decay=0.4)
    t0, t5 = p.perambulator(0), p.perambulator(5)
    assert t0.shape == (256, 256)
    # unit complex variance at t = 0 (re, im ~ N(0, 1/2)), scaled by exp(-0.4 t)
    assert np.mean(np.abs(t0) ** 2) == pytest.approx(1.0, rel=0.02)
    assert np.mean(np.abs(t5) ** 2) == pytest.approx(np.exp(-0.8 * 5), rel=0.02)
    assert abs(np.mean(t0.real * t0.imag)) < 0.01
