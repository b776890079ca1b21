"""Seeded request stream for the solve server: a set of resident meshes of
mixed dimension, order and size, half SIPG Poisson and half LDG
convection-diffusion, and a stream of requests (arrival times, mesh choice,
right-hand side N(0,1) per request).

Meshes: mesh j draws (stream 5, draws 4j .. 4j + 3) a dimension d in {2, 3}
(Poisson) or d = 2 (convection-diffusion, quadrilaterals), an order
p in {1, 2, 3}, a target size log-uniform in [1e3, 2e6] dofs and, for
convection-diffusion, a Peclet number in {1, 100, 1e4}.  The grid has 2^m
cells per side with the m whose dof count is nearest the target in log
scale (and within [1e3, 2e6]), so every aggregate of the bisection hierarchy
has exactly 2^d children.  Candidates: r = the paper's rule (the dof count
of a level-1 aggregate, 2^d elements) capped at 80, the largest r of the
other workloads, which keeps every per-aggregate candidate block of the
setup in shared memory.

Requests: request i picks mesh floor(8 U) (stream 21, draw i), its
inter-arrival gap is -log(1 - U) / rate (stream 37, draw i), and its
right-hand side is N(0,1) from stream 53 + 16 i.

This module holds no arithmetic of the multigrid method.
"""
from dataclasses import dataclass
from typing import List

import numpy as np

from . import rng
from .configs import SEED, convdiff2d, poisson2d, poisson3d

N_MESHES = 8
MIN_DOFS, MAX_DOFS = 1e3, 2e6
R_CAP = 80


@dataclass
class MeshSpec:
    kind: str        # "poisson" or "convdiff"
    dim: int
    p: int
    cells: int       # cells per side (a power of two)
    peclet: float
    dofs: int

    @property
    def name(self):
        pe = f"_pe{self.peclet:g}" if self.kind == "convdiff" else ""
        return f"{self.kind}{self.dim}d_p{self.p}_{self.cells}{pe}"


def _dofs(kind, dim, p, n):
    if kind == "convdiff":
        return n * n * (p + 1) ** 2
    if dim == 2:
        return 2 * n * n * (p + 1) * (p + 2) // 2
    return 6 * n ** 3 * (p + 1) * (p + 2) * (p + 3) // 6


def mesh_specs(seed: int = SEED, count: int = N_MESHES) -> List[MeshSpec]:
    u = rng.uniform(seed, 5, 4 * count)
    out = []
    for j in range(count):
        kind = "poisson" if j < count // 2 else "convdiff"
        dim = (2 if u[4 * j] < 0.5 else 3) if kind == "poisson" else 2
        p = 1 + min(2, int(3 * u[4 * j + 1]))
        target = np.exp(np.log(MIN_DOFS) + u[4 * j + 2] * (np.log(MAX_DOFS) - np.log(MIN_DOFS)))
        best = None
        for m in range(1, 12):
            n = 2 ** m
            d = _dofs(kind, dim, p, n)
            if d < MIN_DOFS or d > MAX_DOFS:
                continue
            err = abs(np.log(d) - np.log(target))
            if best is None or err < best[0]:
                best = (err, n, d)
        if best is None:      # the nearest admissible grid
            n = 2 if _dofs(kind, dim, p, 2) >= MIN_DOFS else 4
            best = (0.0, n, _dofs(kind, dim, p, n))
        pe = [1.0, 100.0, 1e4][min(2, int(3 * u[4 * j + 3]))] if kind == "convdiff" else 0.0
        out.append(MeshSpec(kind, dim, p, best[1], pe, best[2]))
    return out


def build_mesh(spec: MeshSpec, seed: int = SEED):
    """The Problem of one served mesh (levels by the paper's rule)."""
    nb = {"convdiff": (spec.p + 1) ** 2}.get(spec.kind)
    if nb is None:
        nb = ((spec.p + 1) * (spec.p + 2) // 2 if spec.dim == 2
              else (spec.p + 1) * (spec.p + 2) * (spec.p + 3) // 6)
    r = min(2 ** spec.dim * nb, R_CAP)
    if spec.kind == "convdiff":
        return convdiff2d(spec.cells, spec.p, spec.peclet, r=r, seed=seed, name=spec.name)
    if spec.dim == 2:
        return poisson2d(spec.cells, spec.p, r=r, seed=seed, name=spec.name)
    return poisson3d(spec.cells, spec.p, r=r, seed=seed, name=spec.name)


def request_mesh(seed: int, count: int, n_meshes: int = N_MESHES) -> np.ndarray:
    return np.minimum((rng.uniform(seed, 21, count) * n_meshes).astype(np.int64), n_meshes - 1)


def arrival_times(seed: int, count: int, rate: float) -> np.ndarray:
    """Poisson process of the given rate (requests per second)."""
    u = rng.uniform(seed, 37, count)
    return np.cumsum(-np.log1p(-u) / rate)


def request_rhs(seed: int, i: int, n: int) -> np.ndarray:
    return rng.normal(seed, 53 + 16 * i, n)
