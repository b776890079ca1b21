"""Seeded synthetic workloads shaped like the paper's test problems.

Each builder returns a `Problem`: the level-0 operator A (BSR, one dense
n_p x n_p block per pair of face-adjacent elements), the element face graph,
element centroids, the nested aggregate hierarchy (RCB stand-in for METIS),
the right-hand side b ~ N(0,1) per dof (stream 2), the initial candidate
matrix B^0 ~ N(0,1) of n x r entries, column-major (stream 3), and the
solver options the workload fixes.

Workloads (the paper's meshes come from Gmsh/METIS and are not available;
these jittered structured meshes stand in for them):
  poisson2d_p1   32x32 squares, 2 triangles each, SIPG P1 (2048 elements,
                 6144 dofs, 3x3 blocks), levels L0..L3, r = 12, CG.
  poisson2d_p3   256x256, SIPG P3 (131072 elements, 1.31M dofs, 10x10
                 blocks), levels by the paper's rule (L0..L8), r = 4, CG.
  poisson3d_p2   48^3 cubes, 6 Kuhn tets each, SIPG P2 (663552 elements,
                 6.64M dofs, 10x10 blocks), levels L0..L4, r = 80, CG.
  convdiff2d_q2  512x512 quads, LDG diffusion + upwind convection, Q2
                 (262144 elements, 2.36M dofs, 9x9 blocks), GMRES(30).
Any size can be scaled down (n cells per side) for fast tests.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import rng
from .dg import BSR, sipg_assemble
from .hierarchy import chunk_hierarchy, paper_level_count, rcb_order
from .mesh import Mesh, quad_mesh, tet_mesh, tri_mesh

SEED = 13373


@dataclass
class Problem:
    name: str
    mesh: Mesh
    A: BSR
    adj_ptr: np.ndarray
    adj_idx: np.ndarray
    centroids: np.ndarray
    agg_of: List[np.ndarray]          # agg_of[k-1]: level-(k-1) unit -> level-k aggregate
    rhs: np.ndarray
    B0: np.ndarray                     # (n, r) column-major candidates (Fortran order)
    r: int
    solver: str                        # 'cg' or 'gmres'
    dim: int
    p: int
    extra: dict = field(default_factory=dict)

    @property
    def n_levels(self):
        return len(self.agg_of) + 1

    @property
    def n_dofs(self):
        return self.A.n * self.A.b

    def units_per_level(self):
        return [self.A.n] + [int(a.max()) + 1 for a in self.agg_of]


def candidates(seed: int, n: int, r: int) -> np.ndarray:
    """B^0: n x r i.i.d. N(0,1), column j drawn entirely before column j+1."""
    return np.asfortranarray(rng.normal(seed, 3, n * r).reshape(r, n).T)


def rhs(seed: int, n: int) -> np.ndarray:
    return rng.normal(seed, 2, n)


def _finish(name, mesh, A, n_levels, r, solver, p, seed):
    cent = mesh.centroids()
    order = rcb_order(cent)
    aggs = chunk_hierarchy(order, mesh.dim, n_levels)
    ap, ai = mesh.adjacency()
    n = A.n * A.b
    return Problem(name, mesh, A, ap, ai, cent, aggs, rhs(seed, n), candidates(seed, n, r),
                   r, solver, mesh.dim, p)


def poisson2d(n: int = 32, p: int = 1, r: Optional[int] = None, n_levels: Optional[int] = None,
              seed: int = SEED, name: str = "poisson2d") -> Problem:
    mesh = tri_mesh(n, seed, 0.2)
    A = sipg_assemble(mesh, p, 10.0)
    if n_levels is None:
        n_levels = paper_level_count(mesh.n_elems, 2)
    if r is None:
        r = 4 * A.b          # median level-1 aggregate dofs (2^d elements of b dofs)
    return _finish(name, mesh, A, n_levels, r, "cg", p, seed)


def poisson3d(n: int = 48, p: int = 2, r: Optional[int] = None, n_levels: Optional[int] = None,
              seed: int = SEED, name: str = "poisson3d") -> Problem:
    mesh = tet_mesh(n, seed, 0.15)
    A = sipg_assemble(mesh, p, 10.0)
    if n_levels is None:
        n_levels = paper_level_count(mesh.n_elems, 3)
    if r is None:
        r = 8 * A.b
    return _finish(name, mesh, A, n_levels, r, "cg", p, seed)


def poisson2d_p1(seed: int = SEED) -> Problem:
    """32x32 jittered squares, SIPG P1, L0..L3 (3 smoothed levels + dense coarse)."""
    return poisson2d(32, 1, r=12, n_levels=4, seed=seed, name="poisson2d_p1_32x32")


def poisson2d_p3(seed: int = SEED, n: int = 256) -> Problem:
    """256x256 jittered squares, SIPG P3, paper level rule, r = 4."""
    return poisson2d(n, 3, r=4, n_levels=None, seed=seed, name=f"poisson2d_p3_{n}x{n}")


def poisson3d_p2(seed: int = SEED, n: int = 48) -> Problem:
    """48^3 jittered cubes x 6 Kuhn tets, SIPG P2, L0..L4, r = 80."""
    return poisson3d(n, 2, r=80, n_levels=5, seed=seed, name=f"poisson3d_p2_{n}cubed")


def convdiff2d(n: int = 512, p: int = 2, peclet: float = 100.0, r: Optional[int] = None,
               seed: int = SEED, name: Optional[str] = None) -> Problem:
    """n x n jittered quads, LDG diffusion + upwind convection, Q_p, GMRES,
    levels by the paper's rule; r defaults to the level-1 aggregate dofs."""
    from .ldg import ldg_convdiff_assemble
    mesh = quad_mesh(n, seed, 0.2)
    A = ldg_convdiff_assemble(mesh, p, peclet)
    n_levels = paper_level_count(mesh.n_elems, 2)
    if r is None:
        r = 4 * A.b
    if name is None:
        name = f"convdiff2d_q{p}_{n}x{n}_pe{peclet:g}"
    pr = _finish(name, mesh, A, n_levels, r, "gmres", p, seed)
    pr.extra["peclet"] = peclet
    return pr


def convdiff3d(n: int = 16, p: int = 1, peclet: float = 100.0, r: Optional[int] = None,
               seed: int = SEED, name: Optional[str] = None) -> Problem:
    """n^3 jittered cubes x 6 Kuhn tets on the unit cube, LDG diffusion +
    upwind convection with the paper's velocity (1, 2, 3) / sqrt(14), P_p,
    GMRES, levels by the paper's rule; Pe = 0 is pure diffusion, Pe = inf
    pure convection; r defaults to the level-1 aggregate dofs."""
    from .ldg_simplex import ldg_convdiff_simplex
    mesh = tet_mesh(n, seed, 0.15)
    vel = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    A = ldg_convdiff_simplex(mesh, p, peclet, vel)
    n_levels = paper_level_count(mesh.n_elems, 3)
    if r is None:
        r = 8 * A.b
    if name is None:
        name = f"convdiff3d_p{p}_{n}cubed_pe{peclet:g}"
    pr = _finish(name, mesh, A, n_levels, r, "gmres", p, seed)
    pr.extra["peclet"] = peclet
    return pr


def poisson3d_hex(M: int = 4, p: int = 1, r: Optional[int] = None, seed: int = SEED,
                  flux: str = "ip") -> Problem:
    """The paper's first elliptic test (Section 6.1): [-1, 1]^3 cut into 2^M
    hexahedra per side, Q_p, interior penalty (flux='ip', penalty
    (p+1)^2 / h) or minimal-dissipation LDG (flux='ldg'), Dirichlet on
    x = -1 and Neumann elsewhere; the right-hand side is the load vector of
    the manufactured solution exp(sin(pi x) sin(pi y) sin(pi z)) - 1 (not a
    random vector); levels by the paper's rule; r defaults to the level-1
    aggregate dofs."""
    from .hex import hex_mesh, ldg_hex, load_vector, sipg_hex
    mesh = hex_mesh(M)
    A = sipg_hex(mesh, p) if flux == "ip" else ldg_hex(mesh, p)
    n_levels = paper_level_count(mesh.n_elems, 3)
    if r is None:
        r = 8 * A.b
    pr = _finish(f"poisson3d_hex_{flux}_q{p}_M{M}", mesh, A, n_levels, r, "cg", p, seed)
    pr.rhs = load_vector(mesh, p)
    pr.extra["M"] = M
    return pr


def convdiff2d_q2(seed: int = SEED, n: int = 512, peclet: float = 100.0) -> Problem:
    return convdiff2d(n, 2, peclet, r=36, seed=seed)
