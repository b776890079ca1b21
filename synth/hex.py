"""Regular hexahedral meshes of [-1, 1]^3 and the SIPG Poisson problem of the
paper's first elliptic test (Section 6.1), as an input recipe.

Mesh: 2^M hexahedra per side, tensor-product Q_p on each.  Problem:
-Laplace(u) = f with Dirichlet data on the face x = -1 and Neumann data on
the other five faces, manufactured solution
u = exp(sin(pi x) sin(pi y) sin(pi z)) - 1 (zero on x = -1).  SIPG with the
paper's penalty parameter mu = M (p + 1)^2 / 2, read as the face penalty
sigma = mu / h (h the element edge).  The Dirichlet face carries the usual
symmetric boundary terms; Neumann faces enter the right-hand side only.

Elements are numbered e = i + n (j + n k) for the cell (i, j, k); local face
2a is the face at the low end of axis a, 2a + 1 the high end.  No
arithmetic of the multigrid method lives here.
"""
import numpy as np

from .dg import BSR, face_pattern, block_pos, gauss01, tensor_ref
from .mesh import Mesh


def hex_mesh(M: int) -> Mesh:
    n = 2 ** M
    h = 2.0 / n
    ax = -1.0 + h * np.arange(n + 1)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    v0 = i + (n + 1) * (j + (n + 1) * k)
    off = [0, 1, n + 1, n + 2, (n + 1) ** 2, (n + 1) ** 2 + 1, (n + 1) ** 2 + n + 1,
           (n + 1) ** 2 + n + 2]
    elems = np.stack([v0 + o for o in off], axis=1).astype(np.int64)
    e = i + n * (j + n * k)
    ijk = [i, j, k]
    stride = [1, n, n * n]
    inter, bnd = [], []
    for a in range(3):
        m = ijk[a] < n - 1
        inter.append(np.stack([e[m], np.full(m.sum(), 2 * a + 1), e[m] + stride[a],
                               np.full(m.sum(), 2 * a)], axis=1))
        lo = ijk[a] == 0
        hi = ijk[a] == n - 1
        bnd.append(np.stack([e[lo], np.full(lo.sum(), 2 * a)], axis=1))
        bnd.append(np.stack([e[hi], np.full(hi.sum(), 2 * a + 1)], axis=1))
    int_faces = np.concatenate(inter).astype(np.int64)
    bnd_faces = np.concatenate(bnd).astype(np.int64)
    return Mesh("hex", 3, n, h, verts, elems, int_faces, bnd_faces)


def _face_ref(p, a, side):
    """Quadrature on the reference face xi_a = side of [0, 1]^3: points (nq, 3), weights (nq,)."""
    g, w = gauss01(p + 2)
    s, t = np.meshgrid(g, g, indexing="ij")
    ws = np.outer(w, w).ravel()
    other = [c for c in range(3) if c != a]
    xi = np.zeros((s.size, 3))
    xi[:, a] = side
    xi[:, other[0]] = s.ravel()
    xi[:, other[1]] = t.ravel()
    return xi, ws


def sipg_hex(mesh: Mesh, p: int, M: int, dirichlet_faces=((0, 0),)) -> BSR:
    """SIPG for -Laplace on the regular hex mesh; dirichlet_faces lists
    (axis, side) pairs of the domain faces with Dirichlet data (default
    x = -1); the others are Neumann."""
    assert mesh.kind == "hex"
    ref = tensor_ref(3, p)
    nb = ref.nb
    ne = mesh.n_elems
    h = mesh.h
    sigma = M * (p + 1) ** 2 / 2.0 / h
    ptr, col, key = face_pattern(ne, mesh.int_faces)
    val = np.zeros((col.size, nb, nb))
    diag = block_pos(key, ne, np.arange(ne), np.arange(ne))
    # volume: int grad phi_i . grad phi_j = h * int_ref grad_xi phi_i . grad_xi phi_j
    g, w = gauss01(p + 2)
    zq, yq, xq = np.meshgrid(g, g, g, indexing="ij")
    xi = np.stack([xq.ravel(), yq.ravel(), zq.ravel()], axis=1)
    wq = np.einsum("a,b,c->abc", w, w, w).ravel()
    G = ref.grads(xi)
    K = h * np.einsum("q,qid,qjd->ij", wq, G, G)
    val[diag] += K[None]
    area = h * h

    def face_terms(a):
        """phi and d phi / d x_a on the high (side 1) and low (side 0) faces."""
        out = {}
        for side in (0, 1):
            xf, wf = _face_ref(p, a, side)
            out[side] = (ref.values(xf), ref.grads(xf)[..., a] / h, wf * area)
        return out

    for a in range(3):
        ft = face_terms(a)
        F = mesh.int_faces[mesh.int_faces[:, 1] == 2 * a + 1]
        e1, e2 = F[:, 0], F[:, 2]
        ph1, dn1, wf = ft[1]            # element 1 sees the face at its high end; n = +e_a
        ph2, dn2, _ = ft[0]             # element 2 at its low end; same points, same n
        sides = ((ph1, dn1, 1.0), (ph2, dn2, -1.0))
        blocks = {}
        for ia, (pa, da, sa) in enumerate(sides):
            for ib, (pb, db, sb) in enumerate(sides):
                blocks[(ia, ib)] = (-0.5 * sa * np.einsum("q,qi,qj->ij", wf, pa, db)
                                    - 0.5 * sb * np.einsum("q,qi,qj->ij", wf, da, pb)
                                    + sigma * sa * sb * np.einsum("q,qi,qj->ij", wf, pa, pb))
        val[diag[e1]] += blocks[(0, 0)][None]
        val[diag[e2]] += blocks[(1, 1)][None]
        val[block_pos(key, ne, e1, e2)] = blocks[(0, 1)][None]
        val[block_pos(key, ne, e2, e1)] = blocks[(1, 0)][None]
        for side in (0, 1):
            if (a, side) not in dirichlet_faces:
                continue
            B = mesh.bnd_faces[mesh.bnd_faces[:, 1] == 2 * a + side]
            ph, dx, wf = ft[side]
            dn = dx if side == 1 else -dx          # outward normal derivative
            blk = (-np.einsum("q,qi,qj->ij", wf, ph, dn) - np.einsum("q,qi,qj->ij", wf, dn, ph)
                   + sigma * np.einsum("q,qi,qj->ij", wf, ph, ph))
            val[diag[B[:, 0]]] += blk[None]
    return BSR(ne, nb, ptr, col, val)


def exact(x):
    return np.exp(np.prod(np.sin(np.pi * x), axis=-1)) - 1.0


def exact_grad(x):
    s = np.sin(np.pi * x)
    c = np.cos(np.pi * x)
    e = np.exp(np.prod(s, axis=-1))
    return np.stack([np.pi * c[..., 0] * s[..., 1] * s[..., 2] * e,
                     np.pi * s[..., 0] * c[..., 1] * s[..., 2] * e,
                     np.pi * s[..., 0] * s[..., 1] * c[..., 2] * e], axis=-1)


def exact_rhs(x):
    """f = -Laplace(u) for u = exp(S) - 1, S = prod sin(pi x_k)."""
    s = np.sin(np.pi * x)
    c = np.cos(np.pi * x)
    S = np.prod(s, axis=-1)
    e = np.exp(S)
    g = [np.pi * c[..., 0] * s[..., 1] * s[..., 2], np.pi * s[..., 0] * c[..., 1] * s[..., 2],
         np.pi * s[..., 0] * s[..., 1] * c[..., 2]]
    lapS = -3.0 * np.pi ** 2 * S
    return -e * (g[0] ** 2 + g[1] ** 2 + g[2] ** 2 + lapS)


def _element_points(mesh, xi):
    lo = mesh.verts[mesh.elems[:, 0]]
    return lo[:, None, :] + mesh.h * xi[None, :, :]


def load_vector(mesh: Mesh, p: int, dirichlet_faces=((0, 0),)) -> np.ndarray:
    """int_K f phi_i plus the Neumann data int_F (grad u . n) phi_i on the
    non-Dirichlet faces (the Dirichlet data is zero on x = -1)."""
    ref = tensor_ref(3, p)
    g, w = gauss01(p + 4)
    zq, yq, xq = np.meshgrid(g, g, g, indexing="ij")
    xi = np.stack([xq.ravel(), yq.ravel(), zq.ravel()], axis=1)
    wq = np.einsum("a,b,c->abc", w, w, w).ravel() * mesh.h ** 3
    phi = ref.values(xi)
    b = np.einsum("q,eq,qi->ei", wq, exact_rhs(_element_points(mesh, xi)), phi)
    for a in range(3):
        for side in (0, 1):
            if (a, side) in dirichlet_faces:
                continue
            xf, wf = _face_ref(p + 2, a, side)
            B = mesh.bnd_faces[mesh.bnd_faces[:, 1] == 2 * a + side, 0]
            lo = mesh.verts[mesh.elems[B, 0]]
            pts = lo[:, None, :] + mesh.h * xf[None]
            gn = exact_grad(pts)[..., a] * (1.0 if side == 1 else -1.0)
            np.add.at(b, B, np.einsum("q,fq,qi->fi", wf * mesh.h ** 2, gn, ref.values(xf)))
    return b.ravel()


def l2_error(mesh: Mesh, p: int, uh: np.ndarray) -> float:
    ref = tensor_ref(3, p)
    g, w = gauss01(p + 4)
    zq, yq, xq = np.meshgrid(g, g, g, indexing="ij")
    xi = np.stack([xq.ravel(), yq.ravel(), zq.ravel()], axis=1)
    wq = np.einsum("a,b,c->abc", w, w, w).ravel() * mesh.h ** 3
    uq = ref.values(xi) @ uh.reshape(mesh.n_elems, -1).T        # (nq, ne)
    err = (uq.T - exact(_element_points(mesh, xi))) ** 2
    return float(np.sqrt(np.sum(err * wq[None, :])))
