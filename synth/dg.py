"""DG discretisations that produce the test operators (input recipe only).

The paper takes A as given (Section 2, the linear system A u = f of the
DG weak form) and tests interior penalty and LDG fluxes (Section 6).  This
module assembles, in block-sparse row (BSR) form with one dense n_p x n_p
block per pair of face-adjacent elements:

* symmetric interior penalty (SIPG) for -Laplace(u) = f on simplices,
  weak homogeneous Dirichlet data, penalty sigma = c_pen * p^2 / h;
* (see ldg.py for the LDG + upwind convection-diffusion operator on quads).

Basis: nodal Lagrange polynomials at equispaced reference nodes.  It holds
no arithmetic of the multigrid method.
"""
from dataclasses import dataclass
from math import comb

import numpy as np
from numpy.polynomial.legendre import leggauss

from .mesh import Mesh, _simplex_faces


# ----------------------------------------------------------------------------
# reference elements
# ----------------------------------------------------------------------------

def simplex_exponents(dim: int, p: int) -> np.ndarray:
    out = []
    if dim == 2:
        for b in range(p + 1):
            for a in range(p + 1 - b):
                out.append((a, b))
    else:
        for c in range(p + 1):
            for b in range(p + 1 - c):
                for a in range(p + 1 - b - c):
                    out.append((a, b, c))
    return np.array(out, dtype=np.int64)


def tensor_exponents(dim: int, p: int) -> np.ndarray:
    g = np.stack(np.meshgrid(*([np.arange(p + 1)] * dim), indexing="ij"), axis=-1)
    # order: x fastest
    return g.reshape(-1, dim)[:, ::-1].copy() if dim > 1 else g.reshape(-1, 1)


def _powers(xi: np.ndarray, p: int):
    """per coordinate d: (..., p+1) array of xi_d^0 .. xi_d^p"""
    out = []
    for d in range(xi.shape[-1]):
        cols = [np.ones(xi.shape[:-1])]
        for _ in range(p):
            cols.append(cols[-1] * xi[..., d])
        out.append(np.stack(cols, axis=-1))
    return out


def monomials(xi: np.ndarray, ex: np.ndarray) -> np.ndarray:
    """xi (..., d) -> (..., nm): prod_d xi_d^ex[m, d]"""
    pw = _powers(xi, int(ex.max()))
    out = pw[0][..., ex[:, 0]]
    for d in range(1, ex.shape[1]):
        out = out * pw[d][..., ex[:, d]]
    return out


def monomial_grads(xi: np.ndarray, ex: np.ndarray) -> np.ndarray:
    """xi (..., d) -> (..., nm, d)"""
    D = ex.shape[1]
    pw = _powers(xi, int(ex.max()))
    out = np.empty(xi.shape[:-1] + (ex.shape[0], D))
    for k in range(D):
        g = ex[:, k].astype(np.float64) * pw[k][..., np.maximum(ex[:, k] - 1, 0)]
        for d in range(D):
            if d != k:
                g = g * pw[d][..., ex[:, d]]
        out[..., k] = g
    return out


def _wgram(w, a, b):
    """sum_q w[f,q] a[f,q,i] b[f,q,j] -> (f, i, j)"""
    return np.matmul(np.swapaxes(a * w[:, :, None], 1, 2), b)


@dataclass
class RefElement:
    dim: int
    p: int
    ex: np.ndarray       # monomial exponents
    C: np.ndarray        # (nm, nb): basis k = sum_m mono_m * C[m, k]
    nodes: np.ndarray

    @property
    def nb(self):
        return self.C.shape[1]

    def values(self, xi):
        return monomials(xi, self.ex) @ self.C

    def grads(self, xi):
        g = monomial_grads(xi, self.ex)            # (..., nm, d)
        return np.swapaxes(np.matmul(np.swapaxes(g, -1, -2), self.C), -1, -2)


def simplex_ref(dim: int, p: int) -> RefElement:
    ex = simplex_exponents(dim, p)
    nodes = ex.astype(np.float64) / p               # equispaced lattice nodes
    V = monomials(nodes, ex)
    return RefElement(dim, p, ex, np.linalg.inv(V), nodes)


def tensor_ref(dim: int, p: int) -> RefElement:
    ex = tensor_exponents(dim, p)
    nodes = ex.astype(np.float64) / p
    V = monomials(nodes, ex)
    return RefElement(dim, p, ex, np.linalg.inv(V), nodes)


# ----------------------------------------------------------------------------
# quadrature (collapsed Gauss-Legendre on simplices)
# ----------------------------------------------------------------------------

def gauss01(n):
    x, w = leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def simplex_quad(dim: int, degree: int):
    """Points/weights exact for total degree `degree` on the unit simplex."""
    if dim == 1:
        n = degree // 2 + 1
        x, w = gauss01(n)
        return x[:, None], w
    if dim == 2:
        n = (degree + 3) // 2
        u, wu = gauss01(n)
        U, V = np.meshgrid(u, u, indexing="ij")
        W = np.outer(wu, wu)
        x = np.stack([U * (1 - V), V], axis=-1).reshape(-1, 2)
        w = (W * (1 - V)).ravel()
        return x, w
    n = (degree + 4) // 2
    u, wu = gauss01(n)
    U, V, Wc = np.meshgrid(u, u, u, indexing="ij")
    W = wu[:, None, None] * wu[None, :, None] * wu[None, None, :]
    x = np.stack([U * (1 - V) * (1 - Wc), V * (1 - Wc), Wc], axis=-1).reshape(-1, 3)
    w = (W * (1 - V) * (1 - Wc) ** 2).ravel()
    return x, w


# ----------------------------------------------------------------------------
# BSR container and pattern
# ----------------------------------------------------------------------------

@dataclass
class BSR:
    n: int                   # block rows = block cols
    b: int                   # block size
    row_ptr: np.ndarray      # int32 (n+1)
    col: np.ndarray          # int32 (nnzb), sorted per row, diagonal present
    val: np.ndarray          # float64 (nnzb, b, b)

    @property
    def nnzb(self):
        return self.col.size

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.bsr_matrix((self.val, self.col, self.row_ptr),
                             shape=(self.n * self.b, self.n * self.b)).tocsr()


def face_pattern(n_elems: int, int_faces: np.ndarray):
    e1, e2 = int_faces[:, 0], int_faces[:, 2]
    rows = np.concatenate([np.arange(n_elems), e1, e2])
    cols = np.concatenate([np.arange(n_elems), e2, e1])
    o = np.lexsort((cols, rows))
    rows, cols = rows[o], cols[o]
    ptr = np.zeros(n_elems + 1, dtype=np.int64)
    np.add.at(ptr, rows + 1, 1)
    ptr = np.cumsum(ptr)
    key = rows.astype(np.int64) * n_elems + cols
    return ptr.astype(np.int32), cols.astype(np.int32), key


def block_pos(key: np.ndarray, n: int, r, c):
    return np.searchsorted(key, np.asarray(r, np.int64) * n + np.asarray(c, np.int64))


# ----------------------------------------------------------------------------
# SIPG on affine simplices
# ----------------------------------------------------------------------------

def _affine(mesh: Mesh):
    X = mesh.verts[mesh.elems]                           # (ne, d+1, d)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # J[:, :, m] = X_{m+1}-X_0
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    return X, J, det, Jinv


def _face_geometry(mesh, X, e, f):
    """Quadrature points (nF, nq, d), weights*measure (nF, nq), normals (nF, d)
    on local face f of elements e, normal pointing out of e."""
    d = mesh.dim
    lf = np.array(_simplex_faces(d))[f]                  # (nF, d) local vertex ids
    Xe = X[e]                                            # (nF, d+1, d)
    Fv = np.take_along_axis(Xe, lf[:, :, None], axis=1)  # (nF, d, d) face vertices
    return Fv, Xe


def sipg_assemble(mesh: Mesh, p: int, c_pen: float = 10.0, chunk: int = 65536):
    """SIPG operator for -Laplace(u) with weak u = 0 on the boundary.

    a(u, v) = sum_K int_K grad u . grad v
            - sum_F int_F ({grad u}.[[v]] + {grad v}.[[u]])
            + sum_F int_F sigma [[u]].[[v]],   sigma = c_pen p^2 / h
    with [[u]] = u+ n+ + u- n- on interior faces and u n on boundary faces.
    """
    assert mesh.kind in ("tri", "tet")
    d = mesh.dim
    ref = simplex_ref(d, p)
    nb = ref.nb
    ne = mesh.n_elems
    sigma = c_pen * p * p / mesh.h
    X, J, det, Jinv = _affine(mesh)
    assert np.all(det > 0), "inverted element"
    ptr, col, key = face_pattern(ne, mesh.int_faces)
    val = np.zeros((col.size, nb, nb))
    diag = block_pos(key, ne, np.arange(ne), np.arange(ne))

    # volume stiffness: K_e = |det J| sum_q w_q (G_q Jinv)(G_q Jinv)^T
    xq, wq = simplex_quad(d, max(2 * p - 2, 0))
    G = ref.grads(xq)                                     # (nq, nb, d)
    S = np.einsum("q,qia,qjb->ijab", wq, G, G)
    M = np.einsum("eac,ebc->eab", Jinv, Jinv)
    val[diag] += det[:, None, None] * np.einsum("ijab,eab->eij", S, M)

    fx, fw = simplex_quad(d - 1, 2 * p + 1)               # face rule on reference face

    def side_eval(e, xq_phys, nrm):
        """basis values and normal derivatives grad(phi) . n at face points"""
        xi = np.einsum("fkm,fqm->fqk", Jinv[e], xq_phys - X[e][:, None, 0, :])
        phi = ref.values(xi)                              # (nF, nq, nb)
        g = ref.grads(xi)                                 # (nF, nq, nb, d) reference gradients
        jn = np.matmul(Jinv[e], nrm[:, :, None])          # (nF, d, 1): J^{-1} n
        dn = np.matmul(g, jn[:, None, :, :])[..., 0]      # (nF, nq, nb)
        return phi, dn

    def face_points(e, f):
        Fv, Xe = _face_geometry(mesh, X, e, f)
        base = Fv[:, 0, :]
        T = Fv[:, 1:, :] - base[:, None, :]               # (nF, d-1, d)
        pts = base[:, None, :] + np.einsum("qk,fkd->fqd", fx, T)
        if d == 2:
            t = T[:, 0, :]
            meas = np.linalg.norm(t, axis=1)
            nrm = np.stack([t[:, 1], -t[:, 0]], axis=1) / meas[:, None]
            ref_meas = 1.0
        else:
            cr = np.cross(T[:, 0, :], T[:, 1, :])
            meas = np.linalg.norm(cr, axis=1)             # 2 * area
            nrm = cr / meas[:, None]
            ref_meas = 1.0                                # weights already sum to 1/2
        opp = np.take_along_axis(Xe, f[:, None, None].repeat(d, axis=2), axis=1)[:, 0, :]
        flip = np.einsum("fd,fd->f", opp - base, nrm) > 0
        nrm[flip] *= -1.0
        w = fw[None, :] * (meas * ref_meas)[:, None]
        return pts, w, nrm

    # interior faces
    F = mesh.int_faces
    for s in range(0, F.shape[0], chunk):
        e1, f1, e2, f2 = (F[s:s + chunk, c] for c in range(4))
        pts, w, nrm = face_points(e1, f1)
        p1, dn1 = side_eval(e1, pts, nrm)
        p2, dn2 = side_eval(e2, pts, nrm)
        sides = ((p1, dn1, 1.0), (p2, dn2, -1.0))
        blocks = {}
        for a, (pa, dna, sa) in enumerate(sides):
            for b_, (pb, dnb, sb) in enumerate(sides):
                blk = (-0.5 * sa * _wgram(w, pa, dnb)
                       - 0.5 * sb * _wgram(w, dna, pb)
                       + sigma * sa * sb * _wgram(w, pa, pb))
                blocks[(a, b_)] = blk
        # each element has one face per local index, so groups by local face are duplicate-free
        for lf in range(d + 1):
            m1 = f1 == lf
            val[diag[e1[m1]]] += blocks[(0, 0)][m1]
            m2 = f2 == lf
            val[diag[e2[m2]]] += blocks[(1, 1)][m2]
        val[block_pos(key, ne, e1, e2)] = blocks[(0, 1)]
        val[block_pos(key, ne, e2, e1)] = blocks[(1, 0)]

    # boundary faces
    Bf = mesh.bnd_faces
    for s in range(0, Bf.shape[0], chunk):
        e, f = Bf[s:s + chunk, 0], Bf[s:s + chunk, 1]
        pts, w, nrm = face_points(e, f)
        ph, dn = side_eval(e, pts, nrm)
        blk = (-_wgram(w, ph, dn) - _wgram(w, dn, ph) + sigma * _wgram(w, ph, ph))
        for lf in range(d + 1):
            m = f == lf
            val[diag[e[m]]] += blk[m]
    return BSR(ne, nb, ptr, col, val)


def simplex_load_and_error(mesh: Mesh, p: int, f_fun, u_fun=None, u_h=None, degree=None):
    """Load vector int_K f phi_i (and, if u_h is given, the L2 error of the
    DG function u_h against u_fun), by a high-order volume rule."""
    d = mesh.dim
    ref = simplex_ref(d, p)
    X, J, det, Jinv = _affine(mesh)
    deg = degree if degree is not None else 2 * p + 6
    xq, wq = simplex_quad(d, deg)
    phi = ref.values(xq)                                  # (nq, nb)
    xphys = X[:, None, 0, :] + np.einsum("edm,qm->eqd", J, xq)
    if u_h is None:
        fv = f_fun(xphys)                                 # (ne, nq)
        return (det[:, None] * np.einsum("q,eq,qi->ei", wq, fv, phi)).ravel()
    uh = np.einsum("qi,ei->eq", phi, u_h.reshape(mesh.n_elems, -1))
    err = (uh - u_fun(xphys)) ** 2
    return float(np.sqrt(np.sum(det[:, None] * wq[None, :] * err)))


def n_basis(dim: int, p: int, tensor: bool = False) -> int:
    return (p + 1) ** dim if tensor else comb(p + dim, dim)
