"""Batched ensembles on the GPU: graph-captured plans over configurations
with uneven N_v, and the tensor-core kernel variants the autotuner chooses
between, against the oracle and against eager calls."""
import numpy as np
import pytest

from paper_2609_37723_b300 import synth
from oracle import nucleon as orc
from parity import max_c_error, max_c_scaled_error

pytestmark = pytest.mark.gpu

MOM = [(0, 0, 0), (1, 0, 0)]


def T(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def ensemble(nvs, dtype, L=4, nt=3, sigmas=(0.4, 1.1)):
    out = []
    for i, nv in enumerate(nvs):
        p = synth.small(L, nt, nv, mom=MOM, sigmas=sigmas, seed_cfg=100 + i, dtype=dtype)
        out.append((p, p.all_eigvecs(), p.all_perambulators()))
    return out


def device_cfgs(ens, with_lam=True):
    import torch
    cfgs = []
    for p, v, tau in ens:
        c = {"nv": p.nv, "v": T(v), "tau": T(tau), "prof": T(p.prof),
             "C": torch.zeros((p.np_, p.nb, p.nb, p.nt), dtype=torch.complex128, device="cuda")}
        if with_lam:
            c["lam"] = torch.zeros((p.np_, p.nt, p.nb), dtype=torch.complex128, device="cuda")
        cfgs.append(c)
    return cfgs


@pytest.mark.parametrize("autotune", [True, False])
def test_plan_uneven_ensemble_mixed(cuda_lib, autotune):
    from paper_2609_37723_b300 import distil
    ens = ensemble([7, 18, 12], np.complex64)
    cfgs = device_cfgs(ens)
    plan = distil.Plan(4, 3, MOM, 2, 1, "fp16x6", cfgs, autotune=autotune)
    variants, kernels = plan.info()
    assert variants[0] in (0, 1, 2) and variants[1] in (0, 1) and variants[2] in (0, 1)
    assert kernels > 10 * len(cfgs)
    assert distil.get_tuning() == variants
    plan.run()
    plan.stream.synchronize()
    first = [c["C"].cpu().numpy() for c in cfgs]
    for (p, v, tau), c, got in zip(ens, cfgs, first):
        phi = orc.elementals(v.astype(np.complex128), p.L, p.mom)
        ref = orc.correlator(phi, phi[0], tau.astype(np.complex128), p.prof)
        print(f"plan fp16x6 N_v={p.nv}: strict per-entry {max_c_error(got, ref):.2e} "
              f"(scaled {max_c_scaled_error(got, ref):.2e})")
        assert max_c_error(got, ref) < 1e-6, p.nv
        # the same pipeline called eagerly with the plan's kernel variants
        phi_d = distil.elementals(c["v"], p.L, p.mom, "fp16x6")
        eager = distil.correlate(phi_d, phi_d[0], c["tau"], c["prof"], "fp16x6").cpu().numpy()
        assert np.array_equal(eager, got)
        lam = distil.gevp(T(got), 1).cpu().numpy()
        assert np.array_equal(lam, c["lam"].cpu().numpy())
    # a replay of the graph gives the same bytes
    for c in cfgs:
        c["C"].zero_()
    plan.run()
    plan.stream.synchronize()
    for c, got in zip(cfgs, first):
        assert np.array_equal(c["C"].cpu().numpy(), got)
    assert distil.device_status() == 0


def test_tuning_variants_give_identical_results(cuda_lib):
    """Every element accumulates over K in the same order in both kernel
    variants, so switching variants does not change a bit."""
    from paper_2609_37723_b300 import distil
    p = synth.small(4, 2, 20, mom=MOM, sigmas=(0.5, 1.2), seed_cfg=7, dtype=np.complex64)
    v, tau = T(p.all_eigvecs()), T(p.all_perambulators())
    phi = distil.elementals(v, p.L, p.mom, "fp16x6")
    saved = distil.get_tuning()
    try:
        outs = []
        for var in ([0, 0, 0], [1, 1, 1], [1, 0, 1], [2, 0, 1], [2, 1, 0]):
            distil.set_tuning(var)
            outs.append(distil.correlate(phi, phi[0], tau, T(p.prof), "fp16x6").cpu().numpy())
    finally:
        distil.set_tuning(saved)
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_plan_fp64_matches_oracle(cuda_lib):
    from paper_2609_37723_b300 import distil
    ens = ensemble([5, 9], np.complex128, nt=4)
    cfgs = device_cfgs(ens)
    plan = distil.Plan(4, 4, MOM, 2, 2, "fp64", cfgs)
    plan.run()
    plan.stream.synchronize()
    for (p, v, tau), c in zip(ens, cfgs):
        phi = orc.elementals(v, p.L, p.mom)
        ref = orc.correlator(phi, phi[0], tau, p.prof)
        got = c["C"].cpu().numpy()
        assert max_c_scaled_error(got, ref) < 1e-12
        assert np.array_equal(c["lam"].cpu().numpy(), distil.gevp(c["C"], 2).cpu().numpy())
