"""The seeded input recipe: random streams, meshes, SIPG assembly, RCB."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from synth import configs, dg, hierarchy, mesh as M, rng

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))["splitmix64_seed0"]["value"]
    got = [int(v) for v in rng.splitmix64(0, 0, 3)]
    assert got == [int(h, 16) for h in g]


def test_uniform_exact_and_in_range():
    u = rng.uniform(5, 7, 10000)
    assert np.all((u >= 0) & (u < 1))
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))


def test_normal_moments():
    z = rng.normal(3, 3, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01


@pytest.mark.parametrize("n", [3, 8])
def test_tri_mesh_counts(n):
    m = M.tri_mesh(n, 1)
    assert m.n_elems == 2 * n * n
    assert m.int_faces.shape[0] == 3 * n * n - 2 * n      # interior edges
    assert m.bnd_faces.shape[0] == 4 * n
    X = m.verts[m.elems]
    e1, e2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    assert np.all(area > 0) and abs(area.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_tet_mesh_counts(n):
    m = M.tet_mesh(n, 1)
    assert m.n_elems == 6 * n ** 3
    assert m.int_faces.shape[0] == 12 * n ** 3 - 6 * n ** 2
    X = m.verts[m.elems]
    vol = np.einsum("ei,ei->e", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0])) / 6
    assert np.all(vol > 0) and abs(vol.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("n", [1, 5])
def test_tri_mesh_face_graph_closed_form(n):
    """The triangle mesh's face graph in element order, written out by hand:
    square q = j n + i holds triangle 2q (lower right) and 2q + 1 (upper left);
    2q meets 2q + 1, the upper triangle of the square below (2(q - n) + 1) and
    that of the square to the right (2(q + 1) + 1); 2q + 1 meets 2q, the lower
    triangle of the square to the left (2(q - 1)) and that of the square above
    (2(q + n)).  The stand-alone level-0 kernel timing program builds the
    benchmark's block pattern from this rule."""
    m = M.tri_mesh(n, 3)
    ptr, idx = m.adjacency()
    for q in range(n * n):
        i, j = q % n, q // n
        lower = {2 * q + 1} | ({2 * (q - n) + 1} if j > 0 else set()) | \
            ({2 * (q + 1) + 1} if i + 1 < n else set())
        upper = {2 * q} | ({2 * (q - 1)} if i > 0 else set()) | \
            ({2 * (q + n)} if j + 1 < n else set())
        assert set(idx[ptr[2 * q]:ptr[2 * q + 1]].tolist()) == lower
        assert set(idx[ptr[2 * q + 1]:ptr[2 * q + 2]].tolist()) == upper


def test_adjacency_symmetric():
    m = M.tri_mesh(6, 2)
    ptr, idx = m.adjacency()
    pairs = {(i, int(j)) for i in range(m.n_elems) for j in idx[ptr[i]:ptr[i + 1]]}
    assert all((j, i) in pairs for (i, j) in pairs)
    assert max(np.diff(ptr)) == 3


@pytest.mark.parametrize("kind,n,p", [("tri", 6, 1), ("tri", 4, 3), ("tet", 2, 2)])
def test_sipg_symmetric_spd_and_nnzb(kind, n, p):
    m = M.tri_mesh(n, 3) if kind == "tri" else M.tet_mesh(n, 3)
    A = dg.sipg_assemble(m, p)
    S = A.to_scipy()
    assert abs(S - S.T).max() <= 1e-13 * abs(S).max()
    assert sla.eigsh(S, k=1, which="SA", return_eigenvectors=False)[0] > 0
    nfi = m.int_faces.shape[0]
    assert A.nnzb == m.n_elems + 2 * nfi
    assert A.b == dg.n_basis(m.dim, p)


def test_workload_block_counts():
    """nnzb of the 32x32 P1 workload: 2048 + 2 * 3008 (closed form)."""
    pr = configs.poisson2d_p1()
    assert pr.A.nnzb == 8064 and pr.A.b == 3 and pr.n_dofs == 6144


def _u(x):
    return np.exp(np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1])) - 1.0


def _f(x):
    X, Y = x[..., 0], x[..., 1]
    s = np.sin(np.pi * X) * np.sin(np.pi * Y)
    gx = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
    gy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
    return -np.exp(s) * (gx ** 2 + gy ** 2 - 2 * np.pi ** 2 * s)


@pytest.mark.parametrize("p,ns", [(1, (8, 16, 32)), (2, (4, 8, 16)), (3, (4, 8, 16))])
def test_sipg_manufactured_solution_order(p, ns):
    """2D analogue of the paper's manufactured solution (Eq. poissonexact):
    the L2 error falls at order p + 1."""
    errs = []
    for n in ns:
        m = M.tri_mesh(n, 7)
        A = dg.sipg_assemble(m, p).to_scipy()
        b = dg.simplex_load_and_error(m, p, _f)
        uh = sla.spsolve(A.tocsc(), b)
        errs.append(dg.simplex_load_and_error(m, p, _f, _u, uh))
    slope = np.log2(errs[-2] / errs[-1])
    assert slope > p + 1 - 0.2, (errs, slope)


def test_rcb_hand_checked_4x4():
    g = json.load(open(os.path.join(GOLD, "rcb_4x4.json")))
    j, i = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    cent = np.stack([i.ravel() + 0.5, j.ravel() + 0.5], axis=1)
    order = hierarchy.rcb_order(cent)
    assert order.tolist() == g["order"]
    agg = hierarchy.chunk_hierarchy(order, 2, 2)[0]
    groups = [sorted(np.nonzero(agg == a)[0].tolist()) for a in range(4)]
    assert groups == g["level1_aggregates"]


def test_rcb_nesting_sizes_and_relabel_invariance():
    pr = configs.poisson2d(16, 1, r=12, n_levels=4)
    sizes = [np.bincount(a) for a in pr.agg_of]
    assert all(np.all(s == 4) for s in sizes)
    # a relabelling of the elements gives the same aggregates as sets of centroids
    cent = pr.centroids
    perm = np.random.default_rng(0).permutation(cent.shape[0])
    o1 = hierarchy.rcb_order(cent)
    o2 = perm[hierarchy.rcb_order(cent[perm])]
    assert np.array_equal(o1, o2)


def test_paper_level_rule():
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    assert hierarchy.paper_level_count(4096, 3) == g["levels_4096_hex"]["value"]
    assert hierarchy.paper_level_count(131072, 2) == 9


def _quad_load_err(mesh, p, f, uh=None):
    from synth import ldg
    ref = dg.tensor_ref(2, p)
    X = mesh.verts[mesh.elems]
    g, w = dg.gauss01(p + 4)
    S, T = np.meshgrid(g, g, indexing="ij")
    xq = np.stack([S.ravel(), T.ravel()], 1)
    wq = np.outer(w, w).ravel()
    pts, J = ldg._bilinear(X, xq)
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    phi = ref.values(xq)
    if uh is None:
        return np.einsum("eq,eq,qi->ei", wq[None] * det, f(pts), phi).ravel()
    uq = np.einsum("qi,ei->eq", phi, uh.reshape(mesh.n_elems, -1))
    return float(np.sqrt(np.sum(wq[None] * det * (uq - _u(pts)) ** 2)))


@pytest.mark.parametrize("pe,p", [(1.0, 1), (100.0, 2)])
def test_ldg_upwind_manufactured_solution_order(pe, p):
    """LDG diffusion + upwind convection on jittered quads: order p + 1."""
    from synth import ldg
    vel = np.array([np.cos(np.pi / 6), np.sin(np.pi / 6)])

    def f(x):
        X, Y = x[..., 0], x[..., 1]
        s = np.sin(np.pi * X) * np.sin(np.pi * Y)
        gx = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y) * np.exp(s)
        gy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.exp(s)
        lap = np.exp(s) * ((gx / np.exp(s)) ** 2 + (gy / np.exp(s)) ** 2 - 2 * np.pi ** 2 * s)
        return -lap / pe + vel[0] * gx + vel[1] * gy

    errs = []
    for n in (8, 16, 32):
        m = M.quad_mesh(n, 7)
        A = ldg.ldg_convdiff_assemble(m, p, pe)
        uh = sla.spsolve(A.to_scipy().tocsc(), _quad_load_err(m, p, f))
        errs.append(_quad_load_err(m, p, f, uh))
    slope = np.log2(errs[-2] / errs[-1])
    assert slope > p + 1 - 0.2, (errs, slope)


def test_ldg_stencil_and_nonsymmetry():
    """Switch-based LDG couples each element with its 4 face neighbours and
    2 second neighbours (self + 6 in the interior); convection makes A
    nonsymmetric while pure diffusion (no velocity) stays symmetric."""
    from synth import ldg
    m = M.quad_mesh(8, 3)
    A = ldg.ldg_convdiff_assemble(m, 2, 100.0)
    rows = np.diff(A.row_ptr)
    assert rows.max() == 7 and A.b == 9
    S = A.to_scipy()
    assert abs(S - S.T).max() > 1e-3 * abs(S).max()
    Ad = ldg.ldg_convdiff_assemble(m, 2, 1.0, convection=False).to_scipy()
    assert abs(Ad - Ad.T).max() <= 1e-10 * abs(Ad).max()


def _mms_simplex(dim, p, pe, ns, vel):
    from synth.ldg_simplex import ldg_convdiff_simplex
    mu = np.linalg.norm(vel) / pe

    def u(x):
        return np.prod(np.sin(np.pi * x), axis=-1)

    def f(x):
        s = u(x)
        grad = []
        for k in range(dim):
            gk = np.pi * np.cos(np.pi * x[..., k])
            for j in range(dim):
                if j != k:
                    gk = gk * np.sin(np.pi * x[..., j])
            grad.append(gk)
        return mu * dim * np.pi ** 2 * s + sum(vel[k] * grad[k] for k in range(dim))

    errs = []
    for n in ns:
        m = M.tri_mesh(n, 7, 0.2) if dim == 2 else M.tet_mesh(n, 7, 0.15)
        A = ldg_convdiff_simplex(m, p, pe, vel)
        uh = sla.spsolve(A.to_scipy().tocsc(), dg.simplex_load_and_error(m, p, f))
        errs.append(dg.simplex_load_and_error(m, p, f, u, uh))
    return np.log2(errs[-2] / errs[-1]), errs


@pytest.mark.parametrize("dim,p,pe,ns", [(2, 1, 1.0, (8, 16, 32)), (2, 2, 100.0, (8, 16, 32)),
                                         (3, 1, 1.0, (4, 8))])
def test_ldg_simplex_manufactured_solution_order(dim, p, pe, ns):
    """LDG diffusion + upwind convection on triangles and Kuhn tetrahedra:
    the L2 error of u = prod sin(pi x_k) decreases at order p + 1."""
    vel = (np.array([np.cos(np.pi / 6), np.sin(np.pi / 6)]) if dim == 2
           else np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0))
    slope, errs = _mms_simplex(dim, p, pe, ns, vel)
    assert slope > p + 1 - 0.2, (errs, slope)


def test_ldg_simplex_limits_and_structure():
    """Pe = 0 gives the symmetric pure-diffusion LDG operator; Pe = inf the
    pure upwind convection operator, which is block triangular in the flow
    order (no cycles: some ordering makes it block lower triangular), and
    finite Pe their sum with mu = |v| / Pe."""
    from synth.ldg_simplex import ldg_convdiff_simplex
    m = M.tet_mesh(3, 5, 0.15)
    v = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    D = ldg_convdiff_simplex(m, 1, 0.0, v).to_scipy()
    assert abs(D - D.T).max() <= 1e-10 * abs(D).max()
    C = ldg_convdiff_simplex(m, 1, np.inf, v).to_scipy()
    mix = ldg_convdiff_simplex(m, 1, 100.0, v).to_scipy()
    Dv = ldg_convdiff_simplex(m, 1, 1.0, v, convection=False).to_scipy()   # mu = |v| = 1
    assert abs(mix - (C + Dv / 100.0)).max() <= 1e-12 * abs(mix).max()
    # upwind convection couples an element only to its upwind face neighbours
    ne, nb = m.n_elems, 4
    Cb = C.tobsr(blocksize=(nb, nb))
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    pat = sp.csr_matrix((np.ones(Cb.indices.size), Cb.indices, Cb.indptr), shape=(ne, ne))
    pat.setdiag(0)
    pat.eliminate_zeros()
    ncomp, _ = cg.connected_components(pat, directed=True, connection="strong")
    assert ncomp == ne          # no directed cycles between elements


def test_hex_sipg_manufactured_solution_order():
    """The paper's first elliptic test (Section 6.1) on 2^M hexahedra per
    side, Q1, SIPG with face penalty (p+1)^2 / h, Dirichlet on x = -1 and
    Neumann elsewhere: the operator is symmetric positive definite with at
    most 7 blocks per row, and the L2 error of exp(sin sin sin) - 1 falls at
    order p + 1."""
    from synth import hex as HX
    errs = []
    for Mlev in (3, 4):
        m = HX.hex_mesh(Mlev)
        assert HX.hex_penalty(m, 1) == 4.0 / m.h
        A = HX.sipg_hex(m, 1)
        S = A.to_scipy()
        assert abs(S - S.T).max() <= 1e-14 * abs(S).max()
        assert np.diff(A.row_ptr).max() == 7 and A.b == 8
        uh = sla.spsolve(S.tocsc(), HX.load_vector(m, 1))
        errs.append(HX.l2_error(m, 1, uh))
    slope = np.log2(errs[0] / errs[1])
    assert slope > 1.8, (errs, slope)
    m2 = HX.hex_mesh(2)
    assert np.linalg.eigvalsh(HX.sipg_hex(m2, 1).to_scipy().toarray())[0] > 0


def test_hex_ldg_manufactured_solution_order():
    """Minimal-dissipation LDG (switch (1,1,1)) on the same problem: the
    operator is symmetric positive definite, with the compact 7-block
    stencil that a consistent switch gives on a Cartesian mesh, and the L2
    error falls at order p + 1."""
    from synth import hex as HX
    errs = []
    for Mlev in (3, 4):
        m = HX.hex_mesh(Mlev)
        A = HX.ldg_hex(m, 1)
        S = A.to_scipy()
        assert abs(S - S.T).max() <= 1e-13 * abs(S).max()
        assert np.diff(A.row_ptr).max() == 7 and A.b == 8
        uh = sla.spsolve(S.tocsc(), HX.load_vector(m, 1))
        errs.append(HX.l2_error(m, 1, uh))
    slope = np.log2(errs[0] / errs[1])
    assert slope > 1.8, (errs, slope)
    m2 = HX.hex_mesh(2)
    assert np.linalg.eigvalsh(HX.ldg_hex(m2, 1).to_scipy().toarray())[0] > 0


def test_serving_stream_recipe():
    """The request stream of the serving benchmark: eight meshes, the first
    half SIPG Poisson and the rest LDG convection-diffusion on quadrilaterals,
    2^m cells per side, 1e3 - 2e6 dofs, orders 1 - 3, Peclet numbers from
    {1, 100, 1e4}; the dof count formula agrees with the assembled operator on
    the smallest meshes; mesh choices are in range and cover every mesh;
    arrivals are increasing with mean gap 1 / rate."""
    from synth import serving
    specs = serving.mesh_specs(configs.SEED)
    assert len(specs) == serving.N_MESHES
    for j, sp_ in enumerate(specs):
        assert sp_.kind == ("poisson" if j < serving.N_MESHES // 2 else "convdiff")
        assert sp_.cells & (sp_.cells - 1) == 0
        assert serving.MIN_DOFS <= sp_.dofs <= serving.MAX_DOFS
        assert sp_.p in (1, 2, 3)
        assert (sp_.peclet in (1.0, 100.0, 1e4)) == (sp_.kind == "convdiff")
        if sp_.kind == "convdiff":
            assert sp_.dim == 2
    for sp_ in sorted(specs, key=lambda s: s.dofs)[:2]:
        pr = serving.build_mesh(sp_)
        assert pr.n_dofs == sp_.dofs
        assert pr.r <= serving.R_CAP
    which = serving.request_mesh(configs.SEED, 4000)
    assert which.min() >= 0 and which.max() < serving.N_MESHES
    assert set(which.tolist()) == set(range(serving.N_MESHES))
    t = serving.arrival_times(configs.SEED, 4000, 50.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 50.0 - 1.0) < 0.05
    r0, r1 = serving.request_rhs(configs.SEED, 0, 100), serving.request_rhs(configs.SEED, 1, 100)
    assert not np.array_equal(r0, r1)
    assert np.array_equal(r0, serving.request_rhs(configs.SEED, 0, 100))
