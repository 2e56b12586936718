"""Tensor-core (split 16-bit, tcgen05) paths against FP64 references.

Error measures for C (tests/parity.py): the strict per-entry relative error
|dC_ab| / |C_ab| (an entry below 1e-10 of its matrix's largest is measured
against that largest instead), and the error relative to the largest |C_ab|
of its matrix C(p, t) ("scaled").

FP16X6 is the mode that must match the FP64 oracle to 1e-6 per entry: it
splits every row into fixed-point slices (10 + 11 + 11 bits in the mode
contractions, 8 + 11 + 11 with eight products in the elementals) whose
integer products sum exactly in FP32 accumulators of their own, drops
terms below ~5e-9 of the result and keeps double-float arithmetic between
the contractions; its gate is the strict per-entry 1e-6.

The other modes are gated at matrix scale by bounds from their
arithmetic.  BF16X6 (8 + 8 + 8 bits, H = 7): the six kept products drop
mid*lo, lo*mid and lo*lo, of relative size 2^-(W+2+2H) = 2^-24 of the
largest product per term; for rows of random sign this costs about 36 x
that relative to the result (the ratio an emulation of the FP16 split
measures between its dropped-term bound and its error, rows of 4096), so
~2e-6 per contraction.  C passes through five (sink and source
elementals, step i, step j, source): ~5e-6 in quadrature, and an entry at
a quarter of its matrix's largest doubles that at matrix scale: 3e-5.
BF16X3 (8 + 8 bits, 2^-15 per row): ~1.5e-4 per contraction -> 1e-3.
FP16X3 (floating h + l, 22 bits) is limited by the tensor core's FP32
accumulation, which is not correctly rounded (measured ~2.5e-8 per
accumulated MMA): 1e-4.  The strict per-entry errors are printed.
"""
import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth
from parity import max_c_error, max_c_scaled_error, normwise

pytestmark = pytest.mark.gpu

MODES = ["fp16x6", "bf16x6", "bf16x3", "fp16x3"]
TOL_C = {"fp16x6": 1e-6, "fp16x3": 1e-4, "bf16x6": 3e-5, "bf16x3": 1e-3}


def gate(mode, got, ref):
    """The strict per-entry error for FP16X6, the matrix-scale error otherwise."""
    return max_c_error(got, ref) if mode == "fp16x6" else max_c_scaled_error(got, ref)


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
    # the leading slice sums exactly; the second accumulator (about 2^-W |mid/hi|
    # of the result) rounds inexactly, a drift linear in K (the library cuts
    # long contractions into chunks of 4096 for that reason)
    bound = {"fp16x6": 1e-7 + 6e-11 * K, "fp16x3": 3e-8 * max(64, K) * 6 / 16,
             "bf16x6": 1.5e-6 + 1.5e-10 * K, "bf16x3": 3e-4}[mode]
    assert err < bound


@pytest.mark.parametrize("mode", MODES)
def test_correlate_mixed_c1(cuda_lib, mode):
    from paper_2609_37723_b300 import distil
    p = synth.config(1)
    v = p.all_eigvecs().astype(np.complex64)
    tau = p.all_perambulators().astype(np.complex64)
    phi = orc.elementals(v, p.L, p.mom)          # complex128, as the mixed path keeps them
    ref = orc.correlator(phi, phi[0], tau, p.prof)
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), mode).cpu().numpy()
    print(f"correlate {mode} c1: scaled {max_c_scaled_error(got, ref):.2e} strict per-entry "
          f"{max_c_error(got, ref):.2e}")
    assert gate(mode, got, ref) < TOL_C[mode]


@pytest.mark.parametrize("mode", ["fp16x6", "bf16x6"])
@pytest.mark.parametrize("L,nt,nv,nb", [(3, 2, 7, 2), (4, 2, 66, 3), (2, 1, 3, 1), (4, 1, 130, 2)])
def test_correlate_mixed_odd(cuda_lib, mode, L, nt, nv, nb):
    from paper_2609_37723_b300 import distil
    p = synth.small(L, nt, nv, mom=[(0, 0, 0), (1, 1, 0)], sigmas=[0.3, 0.7, 1.4][:nb], seed_cfg=nv + 1,
                    dtype=np.complex64)
    v = p.all_eigvecs()
    tau = p.all_perambulators()
    phi = orc.elementals(v, p.L, p.mom)
    ref = orc.correlator(phi, phi[0], tau, p.prof)
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), mode).cpu().numpy()
    print(f"correlate {mode} L={L} nv={nv}: scaled {max_c_scaled_error(got, ref):.2e} strict "
          f"{max_c_error(got, ref):.2e}")
    assert gate(mode, got, ref) < TOL_C[mode]


# ------------------------------------------------------------------ elementals

TOL_PHI = {"fp16x6": 3e-7, "bf16x6": 3e-6, "bf16x3": 1e-3, "fp16x3": 1e-4}


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,nt,nv,mom", [
    (8, 2, 16, [(0, 0, 0), (1, 0, 0)]),             # workload-1 shape, one K chunk
    (12, 1, 20, [(0, 0, 0), (1, 1, 0), (0, -1, 2)]),  # two K chunks (3 V3 = 5184)
    (3, 2, 7, [(1, 0, 0)]),                          # tiny, ragged everywhere
])
def test_elementals_mixed(cuda_lib, mode, L, nt, nv, mom):
    from paper_2609_37723_b300 import distil
    from parity import phi_error
    p = synth.small(L, nt, nv, mom=mom, seed_cfg=L + nv, dtype=np.complex64)
    v = p.all_eigvecs()
    ref = orc.elementals(v, p.L, p.mom)
    got = distil.elementals(T(v), p.L, p.mom, mode).cpu().numpy()
    assert got.dtype == np.complex128 and got.shape == ref.shape
    e = phi_error(got, ref)
    print(f"elementals {mode} L={L} nv={nv}: {e:.2e}")
    assert e < TOL_PHI[mode]


def test_chain_fp16x6_c1(cuda_lib):
    """Workload 1 end to end on the tensor cores: elementals, correlation
    matrix and GEVP against the FP64 oracle on the same complex64 inputs."""
    from paper_2609_37723_b300 import distil
    p = synth.config(1)
    v = p.all_eigvecs().astype(np.complex64)
    tau = p.all_perambulators().astype(np.complex64)
    ref_phi = orc.elementals(v, p.L, p.mom)
    ref_C = orc.correlator(ref_phi, ref_phi[0], tau, p.prof)
    ph = distil.elementals(T(v), p.L, p.mom, "fp16x6")
    C = distil.correlate(ph, ph[0].contiguous(), T(tau), T(p.prof), "fp16x6")
    e = max_c_error(C.cpu().numpy(), ref_C)
    print(f"chain fp16x6 c1: scaled {max_c_scaled_error(C.cpu().numpy(), ref_C):.2e} strict {e:.2e}")
    assert e < 1e-6


# ------------------------------------------------------------------ boundary checks

def test_misaligned_workspace_rejected(cuda_lib):
    """A workspace that is not 256-byte aligned is refused before any launch,
    and the device status stays clean."""
    import torch
    from paper_2609_37723_b300 import distil
    p = synth.config(1)
    v = p.all_eigvecs().astype(np.complex64)
    tau = p.all_perambulators().astype(np.complex64)
    phi = orc.elementals(v, p.L, p.mom)
    ws_bytes = distil.correlate_workspace(p.nt, p.nv, p.np_, p.nb, "fp16x6")
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(distil.DistilError, match="misaligned"):
        distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), "fp16x6", workspace=ws[16:])
    got = distil.correlate(T(phi), T(phi[0]), T(tau), T(p.prof), "fp16x6", workspace=ws[256:]).cpu().numpy()
    assert max_c_error(got, orc.correlator(phi, phi[0], tau, p.prof)) < TOL_C["fp16x6"]
    assert distil.device_status() == 0
