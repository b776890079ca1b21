"""Jittered structured meshes and their face graphs (input recipe only).

Triangles: the unit square cut into n x n squares, every square split along
the diagonal from (i, j) to (i+1, j+1).  Tetrahedra: the unit cube cut into
n^3 cubes, every cube split into the 6 Kuhn (Freudenthal) tetrahedra that
share the (0,0,0)-(1,1,1) diagonal.  Quadrilaterals: the n x n squares.
Interior vertices move by a seeded uniform jitter of +-a*h per coordinate
(stream 1, vertices in index order, coordinates x, y(, z)).

The face graph is the element adjacency the paper builds its hierarchy on
(Section 4.1: two elements are adjacent when they share a face).
"""
from dataclasses import dataclass
from itertools import permutations

import numpy as np

from . import rng


@dataclass
class Mesh:
    kind: str                 # 'tri', 'tet' or 'quad'
    dim: int
    n: int                    # cells per side
    h: float                  # nominal spacing 1/n
    verts: np.ndarray         # (nv, dim)
    elems: np.ndarray         # (ne, nv_per_elem) int64
    int_faces: np.ndarray     # (nfi, 4): e1, f1, e2, f2 (local face ids)
    bnd_faces: np.ndarray     # (nfb, 2): e, f

    @property
    def n_elems(self) -> int:
        return self.elems.shape[0]

    def centroids(self) -> np.ndarray:
        return self.verts[self.elems].mean(axis=1)

    def adjacency(self):
        """Face graph in CSR form, neighbours sorted by element id."""
        ne = self.n_elems
        e1, e2 = self.int_faces[:, 0], self.int_faces[:, 2]
        src = np.concatenate([e1, e2])
        dst = np.concatenate([e2, e1])
        order = np.lexsort((dst, src))
        src, dst = src[order], dst[order]
        ptr = np.zeros(ne + 1, dtype=np.int64)
        np.add.at(ptr, src + 1, 1)
        return np.cumsum(ptr).astype(np.int32), dst.astype(np.int32)


def _jittered_grid(n: int, dim: int, amp: float, seed: int) -> np.ndarray:
    h = 1.0 / n
    ax = np.arange(n + 1) * h
    if dim == 2:
        yy, xx = np.meshgrid(ax, ax, indexing="ij")       # vertex (i, j) at j*(n+1)+i
        v = np.stack([xx.ravel(), yy.ravel()], axis=1)
        idx = np.arange(n + 1)
        jj, ii = np.meshgrid(idx, idx, indexing="ij")
        interior = ((ii > 0) & (ii < n) & (jj > 0) & (jj < n)).ravel()
    else:
        zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
        v = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
        idx = np.arange(n + 1)
        kk, jj, ii = np.meshgrid(idx, idx, idx, indexing="ij")
        interior = ((ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)).ravel()
    ids = np.nonzero(interior)[0]
    u = rng.uniform(seed, 1, ids.size * dim).reshape(ids.size, dim)
    v[ids] += (2.0 * u - 1.0) * amp * h
    return v


# local faces: face f of a simplex is the one opposite vertex f
def _simplex_faces(dim):
    return [tuple(v for v in range(dim + 1) if v != f) for f in range(dim + 1)]


_QUAD_FACES = [(0, 1), (1, 2), (2, 3), (3, 0)]


def _match_faces(elems: np.ndarray, local_faces):
    ne = elems.shape[0]
    nf = len(local_faces)
    keys = np.stack([np.sort(elems[:, list(lf)], axis=1) for lf in local_faces], axis=1)
    keys = keys.reshape(ne * nf, -1)
    owner = np.repeat(np.arange(ne), nf)
    lface = np.tile(np.arange(nf), ne)
    order = np.lexsort(tuple(keys[:, c] for c in range(keys.shape[1] - 1, -1, -1)))
    ks = keys[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    first = np.nonzero(same)[0]
    a, b = order[first], order[first + 1]
    e1, e2 = owner[a], owner[b]
    f1, f2 = lface[a], lface[b]
    swap = e1 > e2
    e1, e2 = np.where(swap, e2, e1), np.where(swap, e1, e2)
    f1, f2 = np.where(swap, f2, f1), np.where(swap, f1, f2)
    int_faces = np.stack([e1, f1, e2, f2], axis=1)
    o = np.lexsort((e2, e1))
    int_faces = int_faces[o]
    paired = np.zeros(ne * nf, dtype=bool)
    paired[a] = True
    paired[b] = True
    bidx = np.nonzero(~paired)[0]
    bnd = np.stack([owner[bidx], lface[bidx]], axis=1)
    return int_faces.astype(np.int64), bnd.astype(np.int64)


def tri_mesh(n: int, seed: int, amp: float = 0.2) -> Mesh:
    v = _jittered_grid(n, 2, amp, seed)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = j * (n + 1) + i
    v10, v01, v11 = v00 + 1, v00 + (n + 1), v00 + (n + 2)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    elems = np.stack([t1, t2], axis=1).reshape(-1, 3)
    fi, fb = _match_faces(elems, _simplex_faces(2))
    return Mesh("tri", 2, n, 1.0 / n, v, elems, fi, fb)


def tet_mesh(n: int, seed: int, amp: float = 0.15) -> Mesh:
    v = _jittered_grid(n, 3, amp, seed)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = ((k * (n + 1) + j) * (n + 1) + i).ravel()
    step = np.array([1, n + 1, (n + 1) ** 2])
    tets = []
    for perm in permutations(range(3)):
        a = base
        b = a + step[perm[0]]
        c = b + step[perm[1]]
        d = c + step[perm[2]]
        # orientation of the unjittered Kuhn tet follows the permutation parity
        inv = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y])
        t = np.stack([a, b, c, d], axis=1) if inv % 2 == 0 else np.stack([a, c, b, d], axis=1)
        tets.append(t)
    elems = np.stack(tets, axis=1).reshape(-1, 4)
    fi, fb = _match_faces(elems, _simplex_faces(3))
    return Mesh("tet", 3, n, 1.0 / n, v, elems, fi, fb)


def quad_mesh(n: int, seed: int, amp: float = 0.2) -> Mesh:
    v = _jittered_grid(n, 2, amp, seed)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    v00 = (j * (n + 1) + i).ravel()
    elems = np.stack([v00, v00 + 1, v00 + n + 2, v00 + n + 1], axis=1)
    fi, fb = _match_faces(elems, _QUAD_FACES)
    return Mesh("quad", 2, n, 1.0 / n, v, elems, fi, fb)
