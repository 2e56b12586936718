"""Tensor-core (split 16-bit, tcgen05) paths against FP64 references.

Tolerances: FP16x3 and BF16x6 carry 22 and 24 significant bits per operand
and drop cross terms of order 2^-22 / 2^-24, so with FP32 accumulation the
correlation matrix must meet 1e-6 per entry; BF16x3 keeps 16 bits and
drops terms of order 2^-16, gate 1e-4."""
import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth
from parity import max_c_error, normwise

pytestmark = pytest.mark.gpu

MODES = ["fp16x3", "bf16x6", "bf16x3"]
TOL_C = {"fp16x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 1e-4}


def T(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("M,N,K,batch", [(128, 256, 64, 1), (100, 70, 33, 3), (256, 512, 512, 2),
                                         (128, 256, 4096, 1), (128, 256, 32768, 1)])
def test_cgemm_accuracy(cuda_lib, mode, M, N, K, batch):
    from paper_2609_37723_b300 import distil
    rng = np.random.default_rng(M + N + K)
    A = synth.complex_gaussian(rng, (batch, M, K)).astype(np.complex64)
    B = synth.complex_gaussian(rng, (batch, N, K)).astype(np.complex64)
    ref = np.einsum("bmk,bnk->bmn", A.astype(np.complex128), B.astype(np.complex128))
    got = distil.cgemm(T(A), T(B), mode).cpu().numpy()
    err = normwise(got, ref)
    emax = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"cgemm {mode} M={M} N={N} K={K} b={batch}: normwise {err:.2e} max {emax:.2e}")
    bound = {"fp16x3": 2e-6, "bf16x6": 2e-6, "bf16x3": 1e-4}[mode] * max(1.0, np.sqrt(K / 4096))
    assert err < bound


@pytest.mark.parametrize("mode", MODES)
def test_correlate_mixed_c1(cuda_lib, mode):
    from paper_2609_37723_b300 import distil
    p = synth.config(1)
    v = p.all_eigvecs().astype(np.complex64)
    tau = p.all_perambulators().astype(np.complex64)
    phi = orc.elementals(v, p.L, p.mom)
    ref = orc.correlator(phi, phi[0], tau, p.prof)
    ph = phi.astype(np.complex64)
    got = distil.correlate(T(ph), T(ph[0]), T(tau), T(p.prof), mode).cpu().numpy()
    # reference from the same complex64 elementals the GPU sees
    ref64 = orc.correlator(ph, ph[0], tau, p.prof)
    e = max_c_error(got, ref64)
    print(f"correlate {mode} c1: max entry rel err {e:.2e}")
    assert e < TOL_C[mode]


@pytest.mark.parametrize("mode", ["fp16x3", "bf16x6"])
@pytest.mark.parametrize("L,nt,nv,nb", [(3, 2, 7, 2), (4, 2, 66, 3), (2, 1, 3, 1)])
def test_correlate_mixed_odd(cuda_lib, mode, L, nt, nv, nb):
    from paper_2609_37723_b300 import distil
    p = synth.small(L, nt, nv, mom=[(0, 0, 0), (1, 1, 0)], sigmas=[0.3, 0.7, 1.4][:nb], seed_cfg=nv + 1,
                    dtype=np.complex64)
    v = p.all_eigvecs()
    tau = p.all_perambulators()
    phi = orc.elementals(v, p.L, p.mom).astype(np.complex64)
    ref = orc.correlator(phi, phi[0], tau, p.prof)
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), mode).cpu().numpy()
    e = max_c_error(got, ref)
    print(f"correlate {mode} L={L} nv={nv}: {e:.2e}")
    assert e < TOL_C[mode]
