"""Regular hexahedral meshes of [-1, 1]^3 and the SIPG Poisson problem of the
paper's first elliptic test (Section 6.1), as an input recipe.

Mesh: 2^M hexahedra per side, tensor-product Q_p on each.  Problem:
-Laplace(u) = f with Dirichlet data on the face x = -1 and Neumann data on
the other five faces, manufactured solution
u = exp(sin(pi x) sin(pi y) sin(pi z)) - 1 (zero on x = -1).  SIPG with the
paper's penalty parameter, printed as mu = M (p + 1)^2 / 2 (Section 6.1).
It is read as mu = n (p + 1)^2 / 2 with n = 2^M hexahedra per side, i.e.
the exponent of 2^M lost in the printed formula, and mu is the face
penalty itself: since h = 2 / n, mu = (p + 1)^2 / h, the usual 1/h scaling
of an interior-penalty coefficient.  (Reading M as the refinement level and
dividing by h again gives M (p + 1)^2 / (2 h), which grows like log(1/h)/h;
on that reading the oracle needs 11 pCG / 28 stationary iterations at
M = 4 against the paper's 6 / 7, on this one 6 / 9.)  The Dirichlet face
carries the usual symmetric boundary terms; Neumann faces enter the
right-hand side only.

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


def hex_penalty(mesh: Mesh, p: int) -> float:
    """Face penalty mu = n (p + 1)^2 / 2 = (p + 1)^2 / h (n hexahedra per
    side of [-1, 1], h = 2 / n)."""
    return mesh.n * (p + 1) ** 2 / 2.0


def sipg_hex(mesh: Mesh, p: int, dirichlet_faces=((0, 0),)) -> BSR:
    """SIPG for -Laplace on the regular hex mesh; dirichlet_faces lists
    (axis, side) pairs of the domain faces with Dirichlet data (default
    x = -1); the others are Neumann."""
    assert mesh.kind == "hex"
    ref = tensor_ref(3, p)
    nb = ref.nb
    ne = mesh.n_elems
    h = mesh.h
    sigma = hex_penalty(mesh, p)
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


def ldg_hex(mesh: Mesh, p: int, dirichlet_faces=((0, 0),)) -> BSR:
    """Minimal-dissipation LDG for -Laplace on the regular hex mesh (the
    paper's second flux in Section 6.1).  q = grad u is lifted element by
    element: M q^d_K = G^d u_K + sum_F int_F (u_hat - u_K) n_d phi, then
    A u = sum_d [ (G^d)^T q^d - sum_F int_F q_hat_d n_d phi ].  Switch vector
    beta = (1, 1, 1): on an interior face u_hat comes from the element on the
    -beta side (the low one) and q_hat from the +beta side, with no jump
    penalty (C11 = 0).  On a Dirichlet face u_hat = 0 and
    q_hat = q - C11 u n with C11 the face penalty of `hex_penalty`; on a
    Neumann face u_hat = u and q_hat . n is data (right-hand side only).
    The lifted gradients couple an element with neighbours of neighbours,
    so A has a wider block stencil than SIPG; it is symmetric."""
    import scipy.sparse as sp
    assert mesh.kind == "hex"
    ref = tensor_ref(3, p)
    nb = ref.nb
    ne = mesh.n_elems
    h = mesh.h
    C11 = hex_penalty(mesh, p)
    g, w = gauss01(p + 2)
    zq, yq, xq = np.meshgrid(g, g, g, indexing="ij")
    xi = np.stack([xq.ravel(), yq.ravel(), zq.ravel()], axis=1)
    wq = np.einsum("a,b,c->abc", w, w, w).ravel()
    phi = ref.values(xi)
    Gr = ref.grads(xi)
    Mk = h ** 3 * np.einsum("q,qi,qj->ij", wq, phi, phi)
    Minv = np.linalg.inv(Mk)
    Gd = [h ** 2 * np.einsum("q,qi,qj->ij", wq, phi, Gr[..., d]) for d in range(3)]
    area = h * h
    fm = {}
    for a in range(3):
        for side in (0, 1):
            xf, wf = _face_ref(p, a, side)
            fm[(a, side)] = (ref.values(xf), wf * area)

    def fmass(a, s1, s2):
        (p1, wf), (p2, _) = fm[(a, s1)], fm[(a, s2)]
        return np.einsum("q,qi,qj->ij", wf, p1, p2)

    Qr, Qc, Qb = [[] for _ in range(3)], [[] for _ in range(3)], [[] for _ in range(3)]
    Pr, Pc, Pb = [[] for _ in range(3)], [[] for _ in range(3)], [[] for _ in range(3)]
    all_e = np.arange(ne)
    for d in range(3):
        Qr[d].append(all_e); Qc[d].append(all_e)
        Qb[d].append(np.broadcast_to(Minv @ Gd[d], (ne, nb, nb)))
        Pr[d].append(all_e); Pc[d].append(all_e)
        Pb[d].append(np.broadcast_to(Gd[d].T, (ne, nb, nb)))
    for a in range(3):
        F = mesh.int_faces[mesh.int_faces[:, 1] == 2 * a + 1]
        e1, e2 = F[:, 0], F[:, 2]           # e1 low (n = +e_a points into e2), e2 high
        m = e1.size
        F21 = fmass(a, 0, 1)                # e2's face (its low side) x e1's face (high side)
        F22 = fmass(a, 0, 0)
        F12 = fmass(a, 1, 0)
        # lifting of element 2 (outward normal -e_a): int (u1 - u2) (-1) phi
        Qr[a] += [e2, e2]; Qc[a] += [e1, e2]
        Qb[a] += [np.broadcast_to(-Minv @ F21, (m, nb, nb)), np.broadcast_to(Minv @ F22, (m, nb, nb))]
        # primal: q_hat = q2 on both sides; element 1 (n = +e_a), element 2 (n = -e_a)
        Pr[a] += [e1, e2]; Pc[a] += [e2, e2]
        Pb[a] += [np.broadcast_to(-F12, (m, nb, nb)), np.broadcast_to(F22, (m, nb, nb))]
    Dr, Dc, Db = [], [], []
    for a in range(3):
        for side in (0, 1):
            if (a, side) not in dirichlet_faces:
                continue
            B = mesh.bnd_faces[mesh.bnd_faces[:, 1] == 2 * a + side, 0]
            nsign = 1.0 if side == 1 else -1.0
            Fb = fmass(a, side, side)
            # lifting: u_hat = 0 -> int (0 - u) n_a phi
            Qr[a].append(B); Qc[a].append(B)
            Qb[a].append(np.broadcast_to(-nsign * Minv @ Fb, (B.size, nb, nb)))
            # primal: - int (q_hat . n) v with q_hat = q - C11 u n
            Pr[a].append(B); Pc[a].append(B)
            Pb[a].append(np.broadcast_to(-nsign * Fb, (B.size, nb, nb)))
            Dr.append(B); Dc.append(B)
            Db.append(np.broadcast_to(C11 * Fb, (B.size, nb, nb)))

    def block_csr(r, c, b):
        r = np.concatenate(r)
        c = np.concatenate(c)
        b = np.concatenate([np.asarray(x) for x in b])
        ii = (r[:, None, None] * nb + np.arange(nb)[None, :, None]).repeat(nb, axis=2)
        jj = (c[:, None, None] * nb + np.arange(nb)[None, None, :]).repeat(nb, axis=1)
        return sp.csr_matrix((b.ravel(), (ii.ravel(), jj.ravel())), shape=(ne * nb, ne * nb))

    A = block_csr(Dr, Dc, Db) if Dr else sp.csr_matrix((ne * nb, ne * nb))
    for d in range(3):
        A = A + block_csr(Pr[d], Pc[d], Pb[d]) @ block_csr(Qr[d], Qc[d], Qb[d])
    Ab = A.tocsr().tobsr(blocksize=(nb, nb))
    Ab.sort_indices()
    ptr = Ab.indptr.astype(np.int64)
    col = Ab.indices.astype(np.int64)
    rows_of = np.repeat(np.arange(ne), np.diff(ptr))
    assert np.all(np.isin(np.arange(ne), rows_of[col == rows_of]))
    return BSR(ne, nb, ptr.astype(np.int32), col.astype(np.int32), np.ascontiguousarray(Ab.data))


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
