"""Seeded synthetic workloads shaped like the paper's experiments.

This module only generates inputs (mesh sizes, per-node deformation
parameters, initial states, time-step settings).  It holds none of the finite
element arithmetic, so both the CUDA library's tests/benchmark and the CPU
oracle can draw the same inputs from it without sharing any method code.
All random draws use NumPy's ``Generator(PCG64(seed))``.

Configurations (macro mesh NM x NM cells on [0,1]^2, micro mesh Nm x Nm cells
on the reference cell Z = [0,1]^2, Robin edge yhat_1 = 1):

* ``c1``: NM = Nm = 8, Dirichlet macro boundary, bump map with a(x) = 0.1 x_1,
  manufactured sources (``workloads.mms``), dt = 0.01 x 10 steps, FP64,
  CG tolerance 1e-12.
* ``c2``: NM = 64 (4225 micro problems), Nm = 32 (1089 DoFs each), Neumann,
  bump amplitude a ~ U[0, 0.2], D = I, kappa = 1, u0 = 1, v0 = 0,
  dt = 0.005 x 50 steps, relative tolerance 1e-8.
* ``c3``: NM = 128 (16641 problems), Nm = 64 (4225 DoFs), D = diag(1, 0.1),
  shear s ~ U[-0.15, 0.15] and bump b ~ U[0, 0.15], dt = 0.005 x 20 steps.
* ``c4``: 32 independent two-scale problems, NM from {16, 32, 64, 96}, Nm from
  {16, 32, 48}, kappa ~ U[0.5, 2], a(x) = A x_1 x_2 with A ~ U[0, 0.2],
  dt = 0.005 x 10 steps.
* ``c5``: as ``c2`` in FP64 (differentiation workload).

The paper's own experiments use no external dataset; these synthetic inputs
stand in for its convergence and parallel benchmarks.
"""
from __future__ import annotations

import dataclasses

import numpy as np

FAMILY_IDENTITY, FAMILY_BUMP, FAMILY_SHEAR_BUMP, FAMILY_AFFINE, FAMILY_AFFINE_BUMP = 0, 1, 2, 3, 4
NPARAM = {0: 0, 1: 1, 2: 2, 3: 6, 4: 5}


@dataclasses.dataclass
class Workload:
    name: str
    NM: int
    Nm: int
    bc: int                      # 0 Neumann, 1 Dirichlet on the whole macro boundary
    family: int
    params: np.ndarray           # [nM, nparam] (empty for identity)
    D: tuple = (1.0, 0.0, 1.0)   # micro diffusion (D11, D12, D22)
    kappa: float = 1.0
    Du: float = 1.0              # macro diffusion
    dt: float = 0.005
    nsteps: int = 50
    tol: float = 1e-8            # relative residual of the micro / macro solves
    coupling_tol: float = 1e-10
    u0: np.ndarray = None
    v0: np.ndarray = None        # None -> zero

    @property
    def nM(self):
        return (self.NM + 1) ** 2

    @property
    def nm(self):
        return (self.Nm + 1) ** 2

    @property
    def micro_dofs(self):
        return self.nM * self.nm


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def macro_coords(NM: int):
    """(x1, x2) of the macro nodes, node (p, q) -> index p + (NM+1) q."""
    n1 = NM + 1
    k = np.arange(n1 * n1)
    return (k % n1) / NM, (k // n1) / NM


def micro_coords(Nm: int):
    """(yhat1, yhat2) of the reference micro nodes, same numbering."""
    return macro_coords(Nm)


def c1(NM: int = 8, Nm: int = 8) -> Workload:
    x1, _ = macro_coords(NM)
    return Workload("c1", NM, Nm, 1, FAMILY_BUMP, (0.1 * x1).reshape(-1, 1), dt=0.01, nsteps=10,
                    tol=1e-12, coupling_tol=1e-12, u0=None)


def c2(NM: int = 64, Nm: int = 32, seed: int = 0, nsteps: int = 50) -> Workload:
    nM = (NM + 1) ** 2
    a = rng(seed).uniform(0.0, 0.2, nM)
    return Workload("c2", NM, Nm, 0, FAMILY_BUMP, a.reshape(-1, 1), dt=0.005, nsteps=nsteps, tol=1e-8,
                    coupling_tol=1e-10, u0=np.ones(nM))


def c3(NM: int = 128, Nm: int = 64, seed: int = 0, nsteps: int = 20) -> Workload:
    nM = (NM + 1) ** 2
    g = rng(seed)
    s = g.uniform(-0.15, 0.15, nM)
    b = g.uniform(0.0, 0.15, nM)
    return Workload("c3", NM, Nm, 0, FAMILY_SHEAR_BUMP, np.stack([s, b], axis=1), D=(1.0, 0.0, 0.1),
                    dt=0.005, nsteps=nsteps, tol=1e-8, coupling_tol=1e-10, u0=np.ones(nM))


def c4(seed: int = 0, count: int = 32):
    """List of independent two-scale problems of uneven sizes."""
    g = rng(seed)
    out = []
    for k in range(count):
        NM = int(g.choice([16, 32, 64, 96]))
        Nm = int(g.choice([16, 32, 48]))
        kappa = float(g.uniform(0.5, 2.0))
        A = float(g.uniform(0.0, 0.2))
        x1, x2 = macro_coords(NM)
        nM = (NM + 1) ** 2
        out.append(Workload(f"c4[{k}]", NM, Nm, 0, FAMILY_BUMP, (A * x1 * x2).reshape(-1, 1), kappa=kappa,
                            dt=0.005, nsteps=10, tol=1e-8, coupling_tol=1e-10, u0=np.ones(nM)))
    return out


def c5(NM: int = 64, Nm: int = 32, seed: int = 0) -> Workload:
    w = c2(NM, Nm, seed)
    w.name = "c5"
    return w


def random_params(family: int, nM: int, seed: int = 0) -> np.ndarray:
    """Generic seeded parameters of a family, inside the det F > 0 range."""
    g = rng(seed)
    if family == FAMILY_IDENTITY:
        return np.zeros((nM, 0))
    if family == FAMILY_BUMP:
        return g.uniform(0.0, 0.2, (nM, 1))
    if family == FAMILY_SHEAR_BUMP:
        return np.stack([g.uniform(-0.15, 0.15, nM), g.uniform(0.0, 0.15, nM)], axis=1)
    if family == FAMILY_AFFINE:
        A = np.stack([g.uniform(0.8, 1.2, nM), g.uniform(-0.3, 0.3, nM), g.uniform(-0.3, 0.3, nM),
                      g.uniform(0.8, 1.2, nM), g.uniform(-1, 1, nM), g.uniform(-1, 1, nM)], axis=1)
        return A
    if family == FAMILY_AFFINE_BUMP:
        return np.stack([g.uniform(0.8, 1.2, nM), g.uniform(-0.2, 0.2, nM), g.uniform(-0.2, 0.2, nM),
                         g.uniform(0.8, 1.2, nM), g.uniform(0.0, 0.1, nM)], axis=1)
    raise ValueError(family)


def random_state(nM: int, nm: int, seed: int = 1):
    """Seeded smooth-ish initial state (u ~ U[0.5, 1.5], v ~ U[0, 1])."""
    g = rng(seed)
    return g.uniform(0.5, 1.5, nM), g.uniform(0.0, 1.0, nM * nm)
