"""LDG diffusion + upwind convection on affine simplices (input recipe).

-mu Laplace(u) + v . grad(u) = f on the unit square or cube, u = 0 on the
boundary (weakly), mu = |v| L / Pe with L = 1.  Pe = 0 is pure diffusion
(v = 0, mu = 1) and Pe = inf pure convection (mu = 0).  The 3-D workload uses
the paper's velocity v = (1, 2, 3) / sqrt(14) (Section 6.4); its fluxes are
the ones of the quadrilateral recipe (`ldg.py`), written for triangles and
tetrahedra:

* LDG with the switch vector beta = (1, ..., 1): on an interior face u_hat
  comes from the element on the -beta side and q_hat from the +beta side,
  with no jump penalty (C11 = 0); on a boundary face u_hat = 0 and
  q_hat = q - C11 u n with C11 = c_pen p^2 / h;
* q = grad u is eliminated element by element (q in the same space P_p);
* upwind (Godunov) convection: the trace on a face is taken from the element
  the velocity leaves; inflow boundary data is 0.

Blocks are n_p x n_p with n_p = C(p + d, d) (4 for P1 tetrahedra).  No
arithmetic of the multigrid method lives here.
"""
import numpy as np
import scipy.sparse as sp

from .dg import BSR, _affine, _face_geometry, simplex_quad, simplex_ref
from .mesh import Mesh


def _face_points(mesh, X, e, f, fx, fw):
    """Physical quadrature points, weights x measure and unit normals (out of
    element e) on local face f of the elements e."""
    d = mesh.dim
    Fv, Xe = _face_geometry(mesh, X, e, f)
    base = Fv[:, 0, :]
    T = Fv[:, 1:, :] - base[:, None, :]
    pts = base[:, None, :] + np.einsum("qk,fkd->fqd", fx, T)
    if d == 2:
        t = T[:, 0, :]
        meas = np.linalg.norm(t, axis=1)
        nrm = np.stack([t[:, 1], -t[:, 0]], axis=1) / meas[:, None]
    else:
        cr = np.cross(T[:, 0, :], T[:, 1, :])
        meas = np.linalg.norm(cr, axis=1)             # 2 x area; reference weights sum to 1/2
        nrm = cr / meas[:, None]
    opp = np.take_along_axis(Xe, f[:, None, None].repeat(d, axis=2), axis=1)[:, 0, :]
    flip = np.einsum("fd,fd->f", opp - base, nrm) > 0
    nrm[flip] *= -1.0
    return pts, fw[None, :] * meas[:, None], nrm


def ldg_convdiff_simplex(mesh: Mesh, p: int, peclet: float, vel, c_pen: float = 10.0,
                         beta=None, convection: bool = True) -> BSR:
    assert mesh.kind in ("tri", "tet")
    d = mesh.dim
    vel = np.asarray(vel, dtype=np.float64)
    if peclet == 0.0:
        vel = np.zeros(d)
        mu = 1.0
    elif np.isinf(peclet):
        mu = 0.0
    else:
        mu = np.linalg.norm(vel) / peclet
    beta = np.ones(d) if beta is None else np.asarray(beta, dtype=np.float64)
    ref = simplex_ref(d, p)
    nb = ref.nb
    ne = mesh.n_elems
    C11 = c_pen * p * p / mesh.h
    X, J, det, Jinv = _affine(mesh)
    assert np.all(det > 0), "inverted element"

    # ---- volume terms (affine: gradients constant in x for fixed xi) ----
    xq, wq = simplex_quad(d, 2 * p)
    phi = ref.values(xq)                                # (nq, nb)
    gref = ref.grads(xq)                                # (nq, nb, d)
    gphys = np.einsum("qim,emd->eqid", gref, Jinv)      # (ne, nq, nb, d)
    wd = det[:, None] * wq[None, :]                     # (ne, nq)
    Mk = np.einsum("eq,qi,qj->eij", wd, phi, phi)
    Minv = np.linalg.inv(Mk)
    G = [np.einsum("eq,qi,eqj->eij", wd, phi, gphys[..., k]) for k in range(d)]
    vg = np.einsum("eqid,d->eqi", gphys, vel)
    Cvol = -np.einsum("eq,eqi,qj->eij", wd, vg, phi)

    # ---- face terms ----
    fx, fw = simplex_quad(d - 1, 2 * p + 1)

    def side_values(e, pts):
        xi = np.einsum("fkm,fqm->fqk", Jinv[e], pts - X[e][:, None, 0, :])
        return ref.values(xi)                           # (nF, nq, nb)

    rows, cols, blks = [], [], []
    E = mesh.int_faces
    e1, f1, e2 = E[:, 0], E[:, 1], E[:, 2]
    pts, wl, n1 = _face_points(mesh, X, e1, f1, fx, fw)
    p1 = side_values(e1, pts)
    p2 = side_values(e2, pts)
    F11 = np.einsum("fq,fqi,fqj->fij", wl, p1, p1)
    F12 = np.einsum("fq,fqi,fqj->fij", wl, p1, p2)
    F21 = np.einsum("fq,fqi,fqj->fij", wl, p2, p1)
    F22 = np.einsum("fq,fqi,fqj->fij", wl, p2, p2)
    side1_minus = (n1 @ beta) > 0                       # element 1 on the -beta side: u_hat = u1

    Bf = mesh.bnd_faces
    eb, fb = Bf[:, 0], Bf[:, 1]
    ptsb, wlb, nbn = _face_points(mesh, X, eb, fb, fx, fw)
    pb = side_values(eb, ptsb)
    Fbb = np.einsum("fq,fqi,fqj->fij", wlb, pb, pb)

    def block_csr(r, c, b):
        r = np.concatenate(r)
        c = np.concatenate(c)
        b = np.concatenate(b)
        ii = (r[:, None, None] * nb + np.arange(nb)[None, :, None]).repeat(nb, axis=2)
        jj = (c[:, None, None] * nb + np.arange(nb)[None, None, :]).repeat(nb, axis=1)
        return sp.csr_matrix((b.ravel(), (ii.ravel(), jj.ravel())), shape=(ne * nb, ne * nb))

    A = sp.csr_matrix((ne * nb, ne * nb))
    if mu > 0.0:
        # lifted gradient q^k_K = Minv_K [ G^k_K u_K + sum_F (trace - own) n^k ]
        Q = []
        for k in range(d):
            Qr, Qc, Qb = [np.arange(ne)], [np.arange(ne)], [np.einsum("eij,ejk->eik", Minv, G[k])]
            nk = n1[:, k][:, None, None]
            m = side1_minus                             # element 2 sees u_hat = u1, normal -n1
            Qr += [e2[m], e2[m]]
            Qc += [e1[m], e2[m]]
            Qb += [np.einsum("fij,fjk->fik", Minv[e2[m]], -nk[m] * F21[m]),
                   -np.einsum("fij,fjk->fik", Minv[e2[m]], -nk[m] * F22[m])]
            m = ~side1_minus                            # element 1 sees u_hat = u2
            Qr += [e1[m], e1[m]]
            Qc += [e2[m], e1[m]]
            Qb += [np.einsum("fij,fjk->fik", Minv[e1[m]], nk[m] * F12[m]),
                   -np.einsum("fij,fjk->fik", Minv[e1[m]], nk[m] * F11[m])]
            nkb = nbn[:, k][:, None, None]
            Qr.append(eb)
            Qc.append(eb)
            Qb.append(-np.einsum("fij,fjk->fik", Minv[eb], nkb * Fbb))
            Q.append(block_csr(Qr, Qc, Qb))
        # primal rows: sum_k G_k^T q^k - sum_F (q_hat . n_K) traces, + C11 boundary mass
        D = None
        for k in range(d):
            Pr, Pc, Pb = [np.arange(ne)], [np.arange(ne)], [np.transpose(G[k], (0, 2, 1)).copy()]
            nk = n1[:, k][:, None, None]
            m = side1_minus                             # q_hat = q2
            Pr += [e1[m], e2[m]]
            Pc += [e2[m], e2[m]]
            Pb += [-nk[m] * F12[m], nk[m] * F22[m]]
            m = ~side1_minus                            # q_hat = q1
            Pr += [e1[m], e2[m]]
            Pc += [e1[m], e1[m]]
            Pb += [-nk[m] * F11[m], nk[m] * F21[m]]
            nkb = nbn[:, k][:, None, None]
            Pr.append(eb)
            Pc.append(eb)
            Pb.append(-nkb * Fbb)
            term = block_csr(Pr, Pc, Pb) @ Q[k]
            D = term if D is None else D + term
        A = mu * (D + block_csr([eb], [eb], [C11 * Fbb]))

    if convection and np.any(vel != 0.0):
        vn = n1 @ vel
        out1 = vn > 0                                   # flow leaves element 1
        s = vn[:, None, None]
        cr, cc, cb = [np.arange(ne)], [np.arange(ne)], [Cvol]
        cr += [e1[out1], e2[out1]]
        cc += [e1[out1], e1[out1]]
        cb += [s[out1] * F11[out1], -s[out1] * F21[out1]]
        m = ~out1
        cr += [e1[m], e2[m]]
        cc += [e2[m], e2[m]]
        cb += [s[m] * F12[m], -s[m] * F22[m]]
        vb = nbn @ vel
        ob = vb > 0                                     # outflow boundary: interior trace
        cr.append(eb[ob])
        cc.append(eb[ob])
        cb.append(vb[ob][:, None, None] * Fbb[ob])
        A = A + block_csr(cr, cc, cb)
    A = A.tocsr()

    Ab = A.tobsr(blocksize=(nb, nb))
    Ab.sort_indices()
    ptr = Ab.indptr.astype(np.int64)
    col = Ab.indices.astype(np.int64)
    rows_of = np.repeat(np.arange(ne), np.diff(ptr))
    has_diag = np.zeros(ne, bool)
    has_diag[rows_of[col == rows_of]] = True
    assert np.all(has_diag)
    return BSR(ne, nb, ptr.astype(np.int32), col.astype(np.int32), np.ascontiguousarray(Ab.data))
