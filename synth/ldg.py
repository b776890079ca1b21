"""LDG diffusion + upwind convection on bilinear quadrilaterals (input recipe).

-mu Laplace(u) + v . grad(u) = f on the unit square, u = 0 on the boundary
(weakly), v = (cos 30deg, sin 30deg), mu = |v| L / Pe with L = 1.  The paper
uses minimal-dissipation LDG for diffusion and the Godunov (upwind) flux for
convection (Section 6.4); it does not print the fluxes, so this recipe takes
the standard ones:

* LDG with a switch vector beta = (1, 1): on an interior face u_hat comes
  from the element on the -beta side and q_hat from the +beta side, with no
  jump penalty (C11 = 0); on a boundary face u_hat = 0 and
  q_hat = q - C11 u n with C11 = c_pen p^2 / h;
* the auxiliary q = grad u is eliminated element by element (q lives in the
  same tensor space Q_p), so A couples an element with its face neighbours
  and with neighbours of neighbours through the lifted gradients;
* upwind convection: the trace on a face is taken from the element the
  velocity leaves; inflow boundary data is 0.

Blocks are n_p x n_p with n_p = (p+1)^2 (9 for Q2).  No arithmetic of the
multigrid method lives here.
"""
import numpy as np
import scipy.sparse as sp

from .dg import BSR, gauss01, tensor_ref
from .mesh import Mesh

# reference edges of the unit square in the vertex order (0,0),(1,0),(1,1),(0,1):
# edge f runs from vertex f to vertex f+1 (counter-clockwise)
_EDGE = [((0.0, 0.0), (1.0, 0.0)), ((1.0, 0.0), (1.0, 1.0)),
         ((1.0, 1.0), (0.0, 1.0)), ((0.0, 1.0), (0.0, 0.0))]


def _edge_ref(f, t):
    a, b = np.array(_EDGE[f][0]), np.array(_EDGE[f][1])
    return a[None, :] + np.asarray(t)[:, None] * (b - a)[None, :]


def _bilinear(X, xi):
    """X (ne, 4, 2) vertices; xi (nq, 2) -> points (ne, nq, 2), J (ne, nq, 2, 2)."""
    s, t = xi[:, 0], xi[:, 1]
    N = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], axis=1)
    dNs = np.stack([-(1 - t), (1 - t), t, -t], axis=1)
    dNt = np.stack([-(1 - s), -s, s, (1 - s)], axis=1)
    pts = np.einsum("qa,ead->eqd", N, X)
    J = np.stack([np.einsum("qa,ead->eqd", dNs, X), np.einsum("qa,ead->eqd", dNt, X)], axis=-1)
    return pts, J


def ldg_convdiff_assemble(mesh: Mesh, p: int, peclet: float, c_pen: float = 10.0,
                          beta=(1.0, 1.0), vel=None, convection: bool = True) -> BSR:
    assert mesh.kind == "quad"
    if vel is None:
        vel = (np.cos(np.pi / 6), np.sin(np.pi / 6))
    vel = np.asarray(vel, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    mu = np.linalg.norm(vel) * 1.0 / peclet
    ref = tensor_ref(2, p)
    nb = ref.nb
    ne = mesh.n_elems
    X = mesh.verts[mesh.elems]                         # (ne, 4, 2)
    C11 = c_pen * p * p / mesh.h

    # ---- volume terms ----
    g, w = gauss01(p + 3)
    S, T = np.meshgrid(g, g, indexing="ij")
    xq = np.stack([S.ravel(), T.ravel()], axis=1)
    wq = np.outer(w, w).ravel()
    phi = ref.values(xq)                               # (nq, nb)
    gref = ref.grads(xq)                               # (nq, nb, 2)
    _, J = _bilinear(X, xq)                            # (ne, nq, 2, 2)
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    assert np.all(det > 0), "inverted quadrilateral"
    Jinv = np.linalg.inv(J)                            # (ne, nq, 2, 2)
    gphys = np.einsum("qkr,eqrd->eqkd", gref, Jinv)    # (ne, nq, nb, 2)
    wd = wq[None, :] * det                             # (ne, nq)
    Mk = np.einsum("eq,qi,qj->eij", wd, phi, phi)
    Minv = np.linalg.inv(Mk)
    # G^d(i, j) = int phi_i d_d phi_j
    G = [np.einsum("eq,qi,eqj->eij", wd, phi, gphys[..., d]) for d in range(2)]
    # convection volume: -int phi_j (v . grad phi_i)
    vg = np.einsum("eqid,d->eqi", gphys, vel)
    Cvol = -np.einsum("eq,eqi,qj->eij", wd, vg, phi)

    # ---- face geometry ----
    gf, wf = gauss01(p + 3)

    def face_data(e, f, flip):
        a = np.take_along_axis(X[e], f[:, None, None].repeat(2, axis=2), axis=1)[:, 0, :]
        b = np.take_along_axis(X[e], ((f + 1) % 4)[:, None, None].repeat(2, axis=2), axis=1)[:, 0, :]
        tvec = b - a
        length = np.linalg.norm(tvec, axis=1)
        nrm = np.stack([tvec[:, 1], -tvec[:, 0]], axis=1) / length[:, None]   # outward (CCW)
        tt = 1.0 - gf if flip else gf
        vals = np.stack([ref.values(_edge_ref(fi, tt)) for fi in range(4)])   # (4, nfq, nb)
        return vals[f], nrm, length

    # blocks collected as (row elem, col elem, block)
    rows, cols, blks = [], [], []

    def add(r, c, B):
        rows.append(np.asarray(r))
        cols.append(np.asarray(c))
        blks.append(B)

    E = mesh.int_faces
    e1, f1, e2, f2 = E[:, 0], E[:, 1], E[:, 2], E[:, 3]
    p1, n1, L1 = face_data(e1, f1, False)
    p2, _, _ = face_data(e2, f2, True)
    wl = wf[None, :] * L1[:, None]                     # (nF, nfq)
    F11 = np.einsum("fq,fqi,fqj->fij", wl, p1, p1)
    F12 = np.einsum("fq,fqi,fqj->fij", wl, p1, p2)
    F21 = np.einsum("fq,fqi,fqj->fij", wl, p2, p1)
    F22 = np.einsum("fq,fqi,fqj->fij", wl, p2, p2)
    side1_minus = (n1 @ beta) > 0                       # element 1 on the -beta side: u_hat = u1

    # lifted gradient q_K^d = Minv_K [ G^d_K u_K + sum_F (trace-jump terms) ]
    # stored as sparse blocks Q^d (row K, column L)
    Qr, Qc, Qb = [[], []], [[], []], [[], []]
    for d in range(2):
        Qr[d].append(np.arange(ne))
        Qc[d].append(np.arange(ne))
        Qb[d].append(np.einsum("eij,ejk->eik", Minv, G[d]))
    for d in range(2):
        nd = n1[:, d][:, None, None]
        # faces where u_hat = u1 (element 2 takes its neighbour's trace): element 2 gets
        # Minv_2 (E_nbr u1 - E_own u2) with element 2's outward normal -n
        m = side1_minus
        Qr[d] += [e2[m], e2[m]]
        Qc[d] += [e1[m], e2[m]]
        Qb[d] += [np.einsum("fij,fjk->fik", Minv[e2[m]], -nd[m] * F21[m]),
                  -np.einsum("fij,fjk->fik", Minv[e2[m]], -nd[m] * F22[m])]
        # faces where u_hat = u2: element 1 gets Minv_1 (E_nbr u2 - E_own u1)
        m = ~side1_minus
        Qr[d] += [e1[m], e1[m]]
        Qc[d] += [e2[m], e1[m]]
        Qb[d] += [np.einsum("fij,fjk->fik", Minv[e1[m]], nd[m] * F12[m]),
                  -np.einsum("fij,fjk->fik", Minv[e1[m]], nd[m] * F11[m])]
    Bf = mesh.bnd_faces
    eb, fb = Bf[:, 0], Bf[:, 1]
    pb, nbn, Lb = face_data(eb, fb, False)
    wlb = wf[None, :] * Lb[:, None]
    Fbb = np.einsum("fq,fqi,fqj->fij", wlb, pb, pb)
    for d in range(2):
        ndb = nbn[:, d][:, None, None]
        # boundary: u_hat = 0 -> Minv (0 - E_own u_K)
        Qr[d].append(eb)
        Qc[d].append(eb)
        Qb[d].append(-np.einsum("fij,fjk->fik", Minv[eb], ndb * Fbb))

    def block_csr(r, c, b):
        r = np.concatenate(r)
        c = np.concatenate(c)
        b = np.concatenate(b)
        # sum duplicates via scalar COO
        ii = (r[:, None, None] * nb + np.arange(nb)[None, :, None]).repeat(nb, axis=2)
        jj = (c[:, None, None] * nb + np.arange(nb)[None, None, :]).repeat(nb, axis=1)
        return sp.csr_matrix((b.ravel(), (ii.ravel(), jj.ravel())), shape=(ne * nb, ne * nb))

    Q = [block_csr(Qr[d], Qc[d], Qb[d]) for d in range(2)]

    # primal rows: mu [ sum_d G_d^T q^d - sum_F (q_hat . n_K) traces ] + mu C11 boundary mass
    Pr, Pc, Pb = [[], []], [[], []], [[], []]     # operators acting on q^d
    for d in range(2):
        Pr[d].append(np.arange(ne))
        Pc[d].append(np.arange(ne))
        Pb[d].append(np.transpose(G[d], (0, 2, 1)).copy())
        nd = n1[:, d][:, None, None]
        m = side1_minus                              # q_hat = q2
        Pr[d] += [e1[m], e2[m]]
        Pc[d] += [e2[m], e2[m]]
        Pb[d] += [-nd[m] * F12[m], nd[m] * F22[m]]
        m = ~side1_minus                             # q_hat = q1
        Pr[d] += [e1[m], e2[m]]
        Pc[d] += [e1[m], e1[m]]
        Pb[d] += [-nd[m] * F11[m], nd[m] * F21[m]]
        ndb = nbn[:, d][:, None, None]
        Pr[d].append(eb)
        Pc[d].append(eb)
        Pb[d].append(-ndb * Fbb)
    A = None
    for d in range(2):
        term = block_csr(Pr[d], Pc[d], Pb[d]) @ Q[d]
        A = term if A is None else A + term
    A = mu * A + block_csr([eb], [eb], [mu * C11 * Fbb])

    # upwind convection
    vn = n1 @ vel                                    # along element 1's outward normal
    out1 = vn > 0                                    # flow leaves element 1
    cr, cc, cb = [np.arange(ne)], [np.arange(ne)], [Cvol]
    s = vn[:, None, None]
    # trace from element 1 where out1, else from element 2
    cr += [e1[out1], e2[out1]]
    cc += [e1[out1], e1[out1]]
    cb += [s[out1] * F11[out1], -s[out1] * F21[out1]]
    m = ~out1
    cr += [e1[m], e2[m]]
    cc += [e2[m], e2[m]]
    cb += [s[m] * F12[m], -s[m] * F22[m]]
    vb = nbn @ vel
    ob = vb > 0                                      # outflow boundary uses the interior trace
    cr.append(eb[ob])
    cc.append(eb[ob])
    cb.append(vb[ob][:, None, None] * Fbb[ob])
    if convection:
        A = A + block_csr(cr, cc, cb)
    A = A.tocsr()

    # to BSR with the structural block pattern of the stored blocks
    Ab = A.tobsr(blocksize=(nb, nb))
    Ab.sort_indices()
    n = ne
    ptr = Ab.indptr.astype(np.int64)
    col = Ab.indices.astype(np.int64)
    # make sure every diagonal block is stored
    rows_of = np.repeat(np.arange(n), np.diff(ptr))
    has_diag = np.zeros(n, bool)
    has_diag[rows_of[col == rows_of]] = True
    assert np.all(has_diag)
    return BSR(n, nb, ptr.astype(np.int32), col.astype(np.int32), np.ascontiguousarray(Ab.data))
