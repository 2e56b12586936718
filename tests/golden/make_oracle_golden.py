"""Write the stored oracle values the full-size parity tests compare with.

    python tests/golden/make_oracle_golden.py [name ...]

Calls only the FP64 oracle (``oracle/nucleon.py``) and the seeded input
generator (``paper_2609_37723_b300/synth.py``): no value here comes from the
CUDA library.  For each sample below it regenerates the workload's inputs
for the listed timeslices, computes the oracle's source elementals at
t0 = 0 and sink elementals at each sampled t for the sampled momenta, the
whole N_B x N_B matrix C_ab(t) of every sampled (t, p), and the elementals
at a seeded set of triple ranks, and writes them as JSON (complex numbers as
[re, im] pairs) next to this script.  A few raw input values are stored as
well, so a test can check that the inputs it regenerates are the ones the
oracle saw (numpy's generator is bit-reproducible; the orthonormalisation
may differ in the last bit between BLAS builds, far below every tolerance).

The oracle runs at full workload size, so this takes minutes (the largest
sample, L = 48 with N_v = 256, about half an hour on eight cores).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import nucleon as orc  # noqa: E402
from paper_2609_37723_b300 import synth  # noqa: E402

# name -> (workload, configuration, [(t, p), ...])
SAMPLES = {
    # L = 32, N_t = 64, N_v = 128, 5 momenta, 6 profiles: first, second, middle
    # and last timeslice (tau decays as exp(-0.4 t): C spans ~1e-33) at the
    # first and the last momentum
    "L32_Nt64_Nv128": (3, 0, [(t, p) for t in (0, 1, 32, 63) for p in (0, 4)]),
    # one configuration of the uneven ensemble with N_v = 96 (7 momenta)
    "L32_Nt64_cfg3_Nv96": (4, 3, [(t, p) for t in (0, 1, 32, 63) for p in (0, 6)]),
    # two more members of the ensemble, N_v = 128 and 64, first two timeslices
    "L32_Nt64_cfg0_Nv128": (4, 0, [(t, p) for t in (0, 1) for p in (0, 6)]),
    "L32_Nt64_cfg1_Nv64": (4, 1, [(t, p) for t in (0, 1) for p in (0, 6)]),
    # L = 48, N_t = 96, N_v = 256, 9 momenta, 8 profiles: an early slice at
    # p = 0 and the last timeslice at the last momentum
    "L48_Nt96_Nv256": (5, 0, [(1, 0), (95, 8)]),
}
N_PHI_SAMPLES = 64


def cx(a) -> list:
    a = np.asarray(a, dtype=np.complex128)
    return np.stack([a.real, a.imag], axis=-1).tolist()


def make(name: str) -> dict:
    wid, cfg, tps = SAMPLES[name]
    p = synth.config(wid, cfg)
    ts = sorted({t for t, _ in tps})
    ps = sorted({q for _, q in tps})
    mom = p.mom[ps]
    t_start = time.time()
    v0 = p.eigvecs(0).astype(np.complex128)
    src = orc.elementals_t(v0, p.L, mom)                       # [len(ps)][T3]
    out = {"name": name, "workload": wid, "cfg": cfg, "L": p.L, "nt": p.nt, "nv": p.nv, "np": p.np_,
           "nb": p.nb, "samples": [], "inputs": {}}
    rng = np.random.default_rng(2609 + wid)
    ranks = np.sort(rng.choice(p.T3, size=min(N_PHI_SAMPLES, p.T3), replace=False))
    out["phi_ranks"] = ranks.tolist()
    for t in ts:
        vt = v0 if t == 0 else p.eigvecs(t).astype(np.complex128)
        taut = p.perambulator(t)
        snk = src if t == 0 else orc.elementals_t(vt, p.L, mom)
        out["inputs"][str(t)] = {"v_flat": cx(vt.reshape(-1)[:: max(1, vt.size // 8)][:8]),
                                 "tau_flat": cx(taut.reshape(-1)[:: max(1, taut.size // 8)][:8])}
        for t_, q in tps:
            if t_ != t:
                continue
            k = ps.index(q)
            C = orc.correlator_tp(snk[k], src[k], taut.astype(np.complex128), p.prof, p.prof)
            out["samples"].append({"t": t, "p": q, "C": cx(C), "phi": cx(snk[k][ranks])})
            print(f"[golden {name}] t={t} p={q} done at {time.time() - t_start:.0f} s", flush=True)
    out["oracle_seconds"] = time.time() - t_start
    return out


def path_of(name: str) -> str:
    return os.path.join(HERE, f"oracle_{name}.json")


def main(names):
    for name in names or list(SAMPLES):
        data = make(name)
        with open(path_of(name), "w") as f:
            json.dump(data, f)
        print(f"[golden] wrote {path_of(name)}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
