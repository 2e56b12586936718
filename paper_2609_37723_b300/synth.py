"""Seeded synthetic inputs for the distilled-nucleon hot path.

This module holds no arithmetic of the method itself.  It only draws the
random inputs that the elementals and the correlation matrix consume, in the
shapes of the workloads of the nucleon study (distillation with N_v
Laplacian-eigenvector fields per timeslice, perambulators between spin-mode
indices, quark distillation profiles, lattice momenta; Sec. 2.1 of the
paper).  Both the FP64 oracle and the CUDA path read inputs drawn here, so
both see identical bytes.

Conventions (all fixed here, used by every consumer):

* site order  s = x + L*(y + L*z),  x, y, z in 0..L-1;  V3 = L**3.
* eigenvector fields  v[t][i][s][a]  (mode i, site s, colour a fastest);
  the N_v columns of the (3*V3) x N_v matrix with rows (s, a) are an
  orthonormal set (seeded complex Gaussian, orthonormalised by Cholesky-QR).
* perambulators  tau[t][I][I'],  I = alpha*N_v + i  (spin-major), complex
  Gaussian blocks with unit complex variance, scaled by exp(-decay*t).
* profiles  prof[b][i]  real, index form g_i = exp(-(i/N_v)^2 / sigma^2) or
  the index-linear g_i = 1 - i/N_v.
* momenta  mom[q] = integer triples n, p = 2*pi*n/L.

Random streams: numpy PCG64 seeded by SeedSequence(2609, spawn_key=(config,
cfg, t, field)) with field 0 = eigenvectors, 1 = perambulator, 2 = N_v draw,
3 = Laplacian eigenvalues, 4 = gauge links.

Meson workloads (Sec. 2.3 of the paper, "Improved charmonium operators") add
spatial gauge links U[t][k][s][a][b] (direction k = x, y, z; row a, column
b), each an SU(3) matrix drawn from the Haar measure; the covariant
derivatives of the meson operators read them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np
from scipy.linalg import solve_triangular

BASE_SEED = 2609
FIELD_V, FIELD_TAU, FIELD_NV, FIELD_LAMBDA, FIELD_U = 0, 1, 2, 3, 4


def rng_for(config: int, cfg: int, t: int, field: int) -> np.random.Generator:
    ss = np.random.SeedSequence(BASE_SEED, spawn_key=(config, cfg, t, field))
    return np.random.Generator(np.random.PCG64(ss))


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Re, Im ~ N(0, 1/2) independently: unit complex variance."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * math.sqrt(0.5)


def orthonormal_columns(a: np.ndarray) -> np.ndarray:
    """Orthonormalise the columns of a tall complex matrix (Cholesky-QR, twice).

    Q = A R^{-1} with R^H R = A^H A.  A second pass removes the O(u*cond^2)
    loss of orthogonality; for Gaussian A the result is orthonormal to
    rounding.  Any unitary mixing of the columns would do: the consumers read
    the bytes produced here.
    """
    q = a
    for _ in range(2):
        g = q.conj().T @ q
        r = np.linalg.cholesky(g).conj().T  # upper triangular, g = r^H r
        q = solve_triangular(r, q.T, trans="T", lower=False).T  # q r^{-1}
    return q


def haar_su3(rng: np.random.Generator, shape) -> np.ndarray:
    """Haar-distributed SU(3) matrices [*shape][3][3]: QR of a complex
    Gaussian with the phases of R's diagonal moved into Q (Mezzadri's
    recipe for the Haar measure on U(3)), then the determinant's phase
    divided out by a third of it on every entry."""
    z = complex_gaussian(rng, tuple(shape) + (3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q * np.exp(-1j * np.angle(det) / 3.0)[..., None, None]


@dataclasses.dataclass
class Problem:
    """One distillation workload (one gauge configuration)."""
    name: str
    L: int
    nt: int
    nv: int
    mom: np.ndarray          # [np][3] int32
    prof: np.ndarray         # [nb][nv] float64 (t-independent profiles)
    tau_decay: float
    dtype: np.dtype          # complex128 or complex64 storage of v and tau
    config_id: int = 0
    cfg: int = 0

    @property
    def V3(self) -> int:
        return self.L ** 3

    @property
    def np_(self) -> int:
        return int(self.mom.shape[0])

    @property
    def nb(self) -> int:
        return int(self.prof.shape[0])

    @property
    def T3(self) -> int:
        return self.nv * (self.nv - 1) * (self.nv - 2) // 6

    def eigvecs(self, t: int) -> np.ndarray:
        """v[t]: [nv][V3][3] orthonormal over the (site, colour) index."""
        rng = rng_for(self.config_id, self.cfg, t, FIELD_V)
        a = complex_gaussian(rng, (3 * self.V3, self.nv))
        q = orthonormal_columns(a)
        return np.ascontiguousarray(q.T.reshape(self.nv, self.V3, 3)).astype(self.dtype)

    def perambulator(self, t: int) -> np.ndarray:
        """tau[t]: [4nv][4nv] complex Gaussian times exp(-decay*t)."""
        rng = rng_for(self.config_id, self.cfg, t, FIELD_TAU)
        n4 = 4 * self.nv
        return (complex_gaussian(rng, (n4, n4)) * math.exp(-self.tau_decay * t)).astype(self.dtype)

    def laplacian_eigenvalues(self, t: int) -> np.ndarray:
        """Stand-in for the eigenvalues of the N_v lowest modes of the 3D
        Laplacian at timeslice t (the vectors here are random, so any
        increasing positive sequence serves): 0.05 (i+1)^(2/3) times a seeded
        jitter of +-5 %, sorted ascending, float64 [nv]."""
        rng = rng_for(self.config_id, self.cfg, t, FIELD_LAMBDA)
        i = np.arange(self.nv, dtype=np.float64)
        lam = 0.05 * (i + 1.0) ** (2.0 / 3.0) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, self.nv))
        return np.sort(lam)

    def links(self, t: int) -> np.ndarray:
        """U[t]: [3][V3][3][3] spatial gauge links, Haar-random SU(3)."""
        rng = rng_for(self.config_id, self.cfg, t, FIELD_U)
        return haar_su3(rng, (3, self.V3)).astype(self.dtype)

    def all_links(self, ts: Optional[Sequence[int]] = None) -> np.ndarray:
        ts = range(self.nt) if ts is None else ts
        return np.stack([self.links(t) for t in ts])

    def all_eigvecs(self, ts: Optional[Sequence[int]] = None) -> np.ndarray:
        ts = range(self.nt) if ts is None else ts
        return np.stack([self.eigvecs(t) for t in ts])

    def all_perambulators(self, ts: Optional[Sequence[int]] = None) -> np.ndarray:
        ts = range(self.nt) if ts is None else ts
        return np.stack([self.perambulator(t) for t in ts])


def gaussian_profiles(nv: int, sigmas: Sequence[float]) -> np.ndarray:
    i = np.arange(nv, dtype=np.float64)
    return np.stack([np.exp(-((i / nv) ** 2) / (s * s)) for s in sigmas])


def linear_profile(nv: int) -> np.ndarray:
    return 1.0 - np.arange(nv, dtype=np.float64) / nv


MOM_C1 = [(0, 0, 0), (1, 0, 0)]
MOM_C2 = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
MOM_C3 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (1, 1, 1)]
MOM_C4 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
MOM_C5 = MOM_C4 + [(1, 1, 0), (1, 1, 1)]


def _mom(lst) -> np.ndarray:
    return np.asarray(lst, dtype=np.int32).reshape(-1, 3)


def config(cid: int, cfg: int = 0) -> Problem:
    """The five workloads: 1 small FP64, 2 medium, 3 mixed-precision,
    4 batched uneven-N_v ensemble (one member), 5 large."""
    if cid == 1:
        return Problem("L8_Nt8_Nv16", 8, 8, 16, _mom(MOM_C1),
                       gaussian_profiles(16, [0.3, 0.6, 1.0]), 0.5, np.complex128, 1, cfg)
    if cid == 2:
        prof = np.concatenate([gaussian_profiles(64, [0.3, 0.6, 1.0]), linear_profile(64)[None]])
        return Problem("L24_Nt48_Nv64", 24, 48, 64, _mom(MOM_C2), prof, 0.4, np.complex64, 2, cfg)
    if cid == 3:
        sig = [0.2 * 6.0 ** (a / 5.0) for a in range(6)]
        return Problem("L32_Nt64_Nv128", 32, 64, 128, _mom(MOM_C3),
                       gaussian_profiles(128, sig), 0.4, np.complex64, 3, cfg)
    if cid == 4:
        nv = int(rng_for(4, cfg, 0, FIELD_NV).choice([64, 96, 128]))
        sig = [0.2 * 6.0 ** (a / 5.0) for a in range(6)]
        return Problem(f"L32_Nt64_cfg{cfg}_Nv{nv}", 32, 64, nv, _mom(MOM_C4),
                       gaussian_profiles(nv, sig), 0.4, np.complex64, 4, cfg)
    if cid == 5:
        sig = [0.2 * 6.0 ** (a / 7.0) for a in range(8)]
        return Problem("L48_Nt96_Nv256", 48, 96, 256, _mom(MOM_C5),
                       gaussian_profiles(256, sig), 0.4, np.complex64, 5, cfg)
    raise ValueError(f"unknown workload {cid}")


def ensemble4(ncfg: int = 16) -> List[Problem]:
    return [config(4, c) for c in range(ncfg)]


def small(L: int, nt: int, nv: int, mom=MOM_C1, sigmas=(0.3, 0.6, 1.0), decay=0.5,
          dtype=np.complex128, seed_cfg: int = 0) -> Problem:
    """Small problems for tests (config id 0, cfg = seed_cfg)."""
    return Problem(f"L{L}_Nt{nt}_Nv{nv}", L, nt, nv, _mom(mom),
                   gaussian_profiles(nv, sigmas), decay, np.dtype(dtype), 0, seed_cfg)


@dataclasses.dataclass
class MesonProblem:
    """One meson workload: a distillation problem (eigenvectors, links,
    perambulators, momenta, N_B Gaussian profiles per Gamma) plus the size
    of the pruned matrix and the time separation of the pruning SVD."""
    base: Problem
    nkeep: int
    t_prune: int

    def __getattr__(self, name):
        return getattr(self.base, name)


def meson_config(which: str, cfg: int = 0) -> MesonProblem:
    """Meson workloads shaped like the charmonium study (Sec. 2.3: N_f = 2,
    24^3 x 48, N_v = 200, seven Gaussian profiles for each of three Gammas
    giving a 21 x 21 matrix pruned to 8 x 8):
      "charm"  L = 24, N_t = 48, N_v = 200, p = 0, perambulators complex64
               decaying like exp(-0.5 t), profile widths 0.15 .. 1.2
      "small"  L = 8, N_t = 6, N_v = 24, momenta 0 and (0, 0, 1), complex64
      "tiny"   L = 4, N_t = 4, N_v = 6, momenta 0 and (0, 0, 1), complex128
    """
    sig = [0.15 * 8.0 ** (a / 6.0) for a in range(7)]
    if which == "charm":
        base = Problem("L24_Nt48_Nv200_meson", 24, 48, 200, _mom([(0, 0, 0)]),
                       gaussian_profiles(200, sig), 0.5, np.dtype(np.complex64), 6, cfg)
        return MesonProblem(base, 8, 2)
    if which == "small":
        base = Problem("L8_Nt6_Nv24_meson", 8, 6, 24, _mom([(0, 0, 0), (0, 0, 1)]),
                       gaussian_profiles(24, sig), 0.5, np.dtype(np.complex64), 7, cfg)
        return MesonProblem(base, 8, 2)
    if which == "tiny":
        base = Problem("L4_Nt4_Nv6_meson", 4, 4, 6, _mom([(0, 0, 0), (0, 0, 1)]),
                       gaussian_profiles(6, sig), 0.5, np.dtype(np.complex128), 8, cfg)
        return MesonProblem(base, 8, 1)
    raise ValueError(f"unknown meson workload {which}")
