"""End-to-end parity of the CUDA path (setup of Alg. 5, V-cycle of Alg. 2,
CG / GMRES) with the CPU oracle on the same seeded workloads.

Bars: aggregates and sparsity patterns bit-exact; hierarchy values within
1e-8 relative (rounding differences pass through up to 100 relaxation
sweeps and per-aggregate SVDs on every level); iteration counts within +-1;
FP64 solutions within 1e-10 relative of the oracle's; every true residual
<= 1e-10.
"""
import numpy as np
import pytest

from oracle import gasa_oracle as O
from tests.helpers import bsr_scipy, gpu_setup, oracle_setup, problem, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _gasa():
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    return gasa


def level_tolerances(H, base=1e-8):
    """Tolerance of the level-k hierarchy values.  Kept singular vectors move
    by about eps * sigma_1 / gap under rounding (Wedin's bound), gap being
    the distance between the last kept and the first discarded singular
    value; the perturbation then passes through the relaxation and products
    of the levels below, covered by a factor 100.  Aggregates whose last kept
    value is numerically zero use the deterministic completion and do not
    limit the bound."""
    tol, worst = [], base
    for k, L in enumerate(H.levels):
        tol.append(worst)
        if L.svals is None:
            continue
        kept = np.diff(H.levels[k + 1].unit_ptr)
        for sv, s in zip(L.svals, kept):
            if s < sv.size and sv[s - 1] > 1e-10 * sv[0]:
                gap = (sv[s - 1] - sv[s]) / sv[0]
                worst = max(worst, 100 * 2.2e-16 / max(gap, 1e-300))
    return tol


def sparse_rel(G, Ref):
    """max |G - Ref| / max |Ref| over stored entries of either matrix"""
    D = (G - Ref).tocsr()
    d = np.max(np.abs(D.data)) if D.nnz else 0.0
    return d / np.max(np.abs(Ref.data))


def _level_bsr(gasa, ctx, k, which, sh, br, bc, nrows):
    base = {"A": gasa.GASA_LV_A_ROWPTR, "P": gasa.GASA_LV_P_ROWPTR, "R": gasa.GASA_LV_R_ROWPTR}[which]
    nnz = {"A": sh["nnzb"], "P": sh["P_nnzb"], "R": sh["R_nnzb"]}[which]
    rp = gasa.gasa_get_level(ctx, k, base, np.zeros(nrows + 1, np.int32))
    col = gasa.gasa_get_level(ctx, k, base + 1, np.zeros(nnz, np.int32))
    val = gasa.gasa_get_level(ctx, k, base + 2, np.zeros(nnz * br * bc)).reshape(nnz, br, bc)
    return rp, col, val


@pytest.mark.parametrize("name", ["tiny", "c1", "p3_16", "tet_p2_4", "cd_q2_16", "cd3_8_pe100"])
def test_setup_hierarchy(name):
    gasa = _gasa()
    H = oracle_setup(name)
    ctx, info = gpu_setup(name)
    tol = level_tolerances(H)
    try:
        assert info.n_levels == len(H.levels)
        for k, L in enumerate(H.levels):
            sh = gasa.gasa_level_shape(ctx, k)
            sizes = np.diff(L.unit_ptr)
            assert sh["units"] == sizes.size and np.all(sizes == sh["s"])
            assert sh["dofs"] == L.n
            # A_k: pattern bit-exact, values
            rp, col, val = _level_bsr(gasa, ctx, k, "A", sh, sh["s"], sh["s"], sh["units"])
            optr, ocol = O.pattern_csr(L.Apat)
            np.testing.assert_array_equal(rp, optr)
            np.testing.assert_array_equal(col, ocol)
            Ag = bsr_scipy(rp, col, val)
            assert sparse_rel(Ag, L.A) <= tol[k]
            if k == len(H.levels) - 1:
                Ci = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_COARSE_INV, np.zeros(L.n * L.n)).reshape(L.n, L.n)
                assert rel_err(Ci, np.linalg.inv(H.coarse)) <= 100 * tol[k]
                continue
            assert abs(info.rho[k] - L.rho) <= 1e-2 * tol[k] * L.rho
            assert abs(info.omega[k] - L.omega) <= 1e-2 * tol[k] * L.omega
            sw = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_SWEEPS, np.zeros(sh["r"], np.int32))
            np.testing.assert_array_equal(sw, L.sweeps)
            W = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_W, np.zeros(sh["units"] * sh["s"] ** 2))
            assert rel_err(W, L.W.blocks.ravel()) <= tol[k]
            # P: pattern bit-exact, values; R = P^T exactly (same numbers)
            sn = sh["s_next"]
            prp, pcol, pval = _level_bsr(gasa, ctx, k, "P", sh, sh["s"], sn, sh["units"])
            optr, ocol = O.pattern_csr(L.Ppat)
            np.testing.assert_array_equal(prp, optr)
            np.testing.assert_array_equal(pcol, ocol)
            n_next = H.levels[k + 1].unit_ptr.size - 1
            Pg = bsr_scipy(prp, pcol, pval, n_next)
            assert sparse_rel(Pg, L.P) <= tol[k + 1]
            rrp, rcol, rval = _level_bsr(gasa, ctx, k, "R", sh, sn, sh["s"], n_next)
            Rg = bsr_scipy(rrp, rcol, rval, sh["units"])
            assert (Rg - Pg.T).count_nonzero() == 0
    finally:
        gasa.gasa_destroy(ctx)


# dense_tail_dofs: the library default (the coarse levels as one dense
# operator where they are small) and 0 (every coarse step its own launch)
DTAIL = [2048, 0]


@pytest.mark.parametrize("dtail", DTAIL)
@pytest.mark.parametrize("name", ["tiny", "c1", "tet_p2_4", "cd_q2_16", "cd3_4_peinf"])
def test_vcycle(name, dtail):
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    ctx, _ = gpu_setup(name, keep=False, dense_tail_dofs=dtail)
    try:
        M = O.make_vcycle(H)
        want = M(pr.rhs)
        z = to_dev(np.zeros_like(pr.rhs))
        gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z)
        assert rel_err(to_host(z), want) <= 0.1 * level_tolerances(H)[-1]
        Mf = O.make_vcycle(H, "fp32")
        wantf = Mf(pr.rhs)
        gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z, gasa.GASA_PREC_MIXED32)
        assert rel_err(to_host(z), want) <= 1e-4
        assert rel_err(to_host(z), wantf) <= 1e-4
        # FP16 level-0 blocks: same stored values as the oracle's emulation
        # (float32 arithmetic in a different order), and within FP16's
        # resolution of the FP64 cycle
        Mh = O.make_vcycle(H, "fp16")
        wanth = Mh(pr.rhs)
        gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z, gasa.GASA_PREC_MIXED16)
        assert rel_err(to_host(z), wanth) <= 1e-4
        assert rel_err(to_host(z), want) <= 1e-2
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("dtail", DTAIL)
@pytest.mark.parametrize("name", ["tiny", "c1", "p3_16", "tet_p2_4"])
def test_cg_solve(name, dtail):
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    ref = O.solve(H, pr.rhs, TOL, "cg", max_iter=5000)
    ref32 = O.solve(H, pr.rhs, TOL, "cg", precision="mixed32", max_iter=5000)
    ctx, _ = gpu_setup(name, keep=False, dense_tail_dofs=dtail)
    try:
        x = np.zeros_like(pr.rhs)
        info = gasa.gasa_solve(ctx, pr.rhs, x, TOL)
        assert info.converged and info.rel_residual <= TOL
        assert abs(info.iterations - ref.iterations) <= 1, (info.iterations, ref.iterations)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= TOL
        xm = np.zeros_like(pr.rhs)
        info32 = gasa.gasa_solve(ctx, pr.rhs, xm, TOL, gasa.GASA_PREC_MIXED32)
        assert info32.converged and info32.rel_residual <= TOL
        assert abs(info32.iterations - ref32.iterations) <= 1, (info32.iterations, ref32.iterations)
        ref16 = O.solve(H, pr.rhs, TOL, "cg", precision="mixed16", max_iter=5000)
        xh = np.zeros_like(pr.rhs)
        info16 = gasa.gasa_solve(ctx, pr.rhs, xh, TOL, gasa.GASA_PREC_MIXED16)
        assert info16.converged and info16.rel_residual <= TOL
        assert abs(info16.iterations - ref16.iterations) <= 1, (info16.iterations, ref16.iterations)
        # device-resident buffers give the same answer
        xd = to_dev(np.zeros_like(pr.rhs))
        info_d = gasa.gasa_solve(ctx, to_dev(pr.rhs), xd, TOL, on_device=True)
        assert info_d.iterations == info.iterations
        assert np.max(np.abs(to_host(xd) - x)) == 0.0
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("name", ["tiny", "c1", "cd_q2_16", "cd_q2_32_pe1e4", "cd_q2_32_pe1",
                                  "cd3_4_pe0", "cd3_4_pe1000", "cd3_4_peinf", "cd3_8_pe100"])
def test_gmres_solve(name):
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    ref = O.solve(H, pr.rhs, TOL, "gmres", restart=30, max_iter=5000)
    ref32 = O.solve(H, pr.rhs, TOL, "gmres", precision="mixed32", restart=30, max_iter=5000)
    ctx, _ = gpu_setup(name, keep=False, solver=1)
    try:
        x = np.zeros_like(pr.rhs)
        info = gasa.gasa_solve(ctx, pr.rhs, x, TOL)
        assert info.converged and info.rel_residual <= TOL
        assert abs(info.iterations - ref.iterations) <= 1, (info.iterations, ref.iterations)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-9
        xm = np.zeros_like(pr.rhs)
        info32 = gasa.gasa_solve(ctx, pr.rhs, xm, TOL, gasa.GASA_PREC_MIXED32)
        assert info32.converged and info32.rel_residual <= TOL
        assert abs(info32.iterations - ref32.iterations) <= 1, (info32.iterations, ref32.iterations)
        ref16 = O.solve(H, pr.rhs, TOL, "gmres", precision="mixed16", restart=30, max_iter=5000)
        info16 = gasa.gasa_solve(ctx, pr.rhs, xm, TOL, gasa.GASA_PREC_MIXED16)
        assert info16.converged and info16.rel_residual <= TOL
        assert abs(info16.iterations - ref16.iterations) <= 1, (info16.iterations, ref16.iterations)
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("name", ["p3_16", "p3_32"])
def test_bulk_staged_sweep_same_bits(name):
    """The level-0 FP32 smoothing step with bulk-copy staging computes the
    same operations in the same order as the unstaged plain step (the folded
    step is off on both sides): the solves agree bit for bit (10x10 blocks
    qualify for staging)."""
    gasa = _gasa()
    pr = problem(name)
    out = []
    for staging in (1, 0):
        ctx, _ = gpu_setup(name, keep=False, bulk_staging=staging, folded_smoother=0)
        try:
            x = np.zeros_like(pr.rhs)
            info = gasa.gasa_solve(ctx, pr.rhs, x, TOL, gasa.GASA_PREC_MIXED32)
            z = to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z, gasa.GASA_PREC_MIXED32)
            out.append((info.iterations, x, to_host(z)))
        finally:
            gasa.gasa_destroy(ctx)
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("name", ["c1", "p3_16"])
def test_graph_solve_equals_host_loop(name):
    """The CG loop captured in one CUDA graph (device-side stopping test)
    runs the same kernels in the same order as the host-driven loop, so the
    iterates agree bit for bit."""
    gasa = _gasa()
    pr = problem(name)
    ctx, _ = gpu_setup(name, keep=False)
    try:
        for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32):
            xg = np.zeros_like(pr.rhs)
            ig = gasa.gasa_solve(ctx, pr.rhs, xg, TOL, prec)
            gasa.gasa_profile_enable(ctx, True)          # profiling selects the host-driven loop
            xh = np.zeros_like(pr.rhs)
            ih = gasa.gasa_solve(ctx, pr.rhs, xh, TOL, prec)
            gasa.gasa_profile_enable(ctx, False)
            assert ig.iterations == ih.iterations
            assert np.array_equal(xg, xh)
            # solving twice gives the same bits (deterministic reductions)
            xg2 = np.zeros_like(pr.rhs)
            gasa.gasa_solve(ctx, pr.rhs, xg2, TOL, prec)
            assert np.array_equal(xg, xg2)
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_stationary_solve(name):
    """Alg. 2 as a solver (x <- x + V(b - A x)) in FP64 and with the FP32
    V-cycle (iterative refinement): iteration counts within 1 of the oracle,
    FP64 solution within 1e-10; graph and host-driven loops agree bit for bit."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    ref = O.stationary(H, pr.rhs, TOL, max_iter=1000)
    ref32 = O.stationary(H, pr.rhs, TOL, max_iter=1000, precision="mixed32")
    assert ref.converged and ref32.converged
    ctx, _ = gpu_setup(name, keep=False, solver=gasa.GASA_SOLVER_STATIONARY)
    try:
        x = np.zeros_like(pr.rhs)
        info = gasa.gasa_solve(ctx, pr.rhs, x, TOL)
        assert info.converged and info.rel_residual <= TOL
        assert abs(info.iterations - ref.iterations) <= 1, (info.iterations, ref.iterations)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= TOL
        xm = np.zeros_like(pr.rhs)
        info32 = gasa.gasa_solve(ctx, pr.rhs, xm, TOL, gasa.GASA_PREC_MIXED32)
        assert info32.converged and info32.rel_residual <= TOL
        assert abs(info32.iterations - ref32.iterations) <= 1, (info32.iterations, ref32.iterations)
        gasa.gasa_profile_enable(ctx, True)
        xh = np.zeros_like(pr.rhs)
        ih = gasa.gasa_solve(ctx, pr.rhs, xh, TOL)
        gasa.gasa_profile_enable(ctx, False)
        assert ih.iterations == info.iterations
        assert np.array_equal(xh, x)
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("name,kappa", [("c1", 1), ("c1", 2), ("cd_q2_16", 2), ("p3_16", 3)])
def test_matrix_free_levels(name, kappa):
    """Section 4.4: A_1 .. A_kappa dropped after setup and applied through the
    transfers.  The V-cycle matches the oracle's matrix-free V-cycle, the
    solves match the oracle's (iterations within 1, FP64 solution within
    1e-10), the stored A_k are gone and the resident hierarchy is smaller."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    # the resident hierarchy is compared without the dense bottom operator,
    # whose size depends on the first level it can start from
    ctx0, info0 = gpu_setup(name, keep=False, dense_tail_dofs=0)
    ctxm, infom = gpu_setup(name, keep=False, matrix_free_levels=kappa, dense_tail_dofs=0)
    gasa.gasa_destroy(ctxm)
    ctx, info = gpu_setup(name, keep=False, matrix_free_levels=kappa)
    try:
        assert infom.device_bytes < info0.device_bytes
        want = O.make_vcycle(H, matrix_free_levels=kappa)(pr.rhs)
        z = to_dev(np.zeros_like(pr.rhs))
        gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z)
        assert rel_err(to_host(z), want) <= 0.1 * level_tolerances(H)[-1]
        wantf = O.make_vcycle(H, "fp32", matrix_free_levels=kappa)(pr.rhs)
        gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z, gasa.GASA_PREC_MIXED32)
        assert rel_err(to_host(z), wantf) <= 1e-4
        solver = pr.solver
        ref = O.solve(H, pr.rhs, TOL, solver, restart=30, max_iter=5000, matrix_free_levels=kappa)
        x = np.zeros_like(pr.rhs)
        inf = gasa.gasa_solve(ctx, pr.rhs, x, TOL)
        assert inf.converged and inf.rel_residual <= TOL
        assert abs(inf.iterations - ref.iterations) <= 1, (inf.iterations, ref.iterations)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= TOL
        ref32 = O.solve(H, pr.rhs, TOL, solver, precision="mixed32", restart=30, max_iter=5000,
                        matrix_free_levels=kappa)
        inf32 = gasa.gasa_solve(ctx, pr.rhs, x, TOL, gasa.GASA_PREC_MIXED32)
        assert inf32.converged and abs(inf32.iterations - ref32.iterations) <= 1
        for k in range(1, kappa + 1):
            with pytest.raises(gasa.GasaError):
                gasa.gasa_get_level(ctx, k, gasa.GASA_LV_A_VAL, np.zeros(1))
        # the request server runs matrix-free levels too
        srv = gasa.gasa_server_create(0, 8 << 30, 4)
        try:
            mid = gasa.gasa_server_add_mesh(srv, ctx)
            t = gasa.gasa_server_submit(srv, mid, pr.rhs, TOL, gasa.GASA_PREC_FP64)
            gasa.gasa_server_drain(srv, 300.0)
            xs = np.zeros_like(pr.rhs)
            st, si = gasa.gasa_server_poll(srv, t, xs)
            assert st == gasa.GASA_OK and si.rel_residual <= TOL
            assert abs(si.iterations - ref.iterations) <= 1
            assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= TOL
        finally:
            gasa.gasa_server_destroy(srv)
    finally:
        gasa.gasa_destroy(ctx)
        gasa.gasa_destroy(ctx0)


@pytest.mark.parametrize("name", ["hex_M3", "hex_M4", "hexldg_M3", "hexldg_M4"])
def test_paper_hex_poisson(name):
    """The paper's first elliptic test (Section 6.1) at M = 3 and 4 (4,096 and
    32,768 dofs, Q1 hexahedra, IP or LDG flux, mixed Dirichlet/Neumann,
    manufactured right-hand side, tol 1e-7): CG-preconditioned and
    stationary solves match the oracle's iteration counts within 1, and the
    GPU counts sit in the band of the paper's table (pCG within 1 of the
    paper's, stationary at most 3 above it, 4 with the GPU's own +-1)."""
    import json, os
    table = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_hex_table.json")))
    flux = "ldg" if name.startswith("hexldg") else "ip"
    M = name.split("_M")[1]
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    tol = 1e-7
    ref_cg = O.solve(H, pr.rhs, tol, "cg", max_iter=500)
    ref_st = O.stationary(H, pr.rhs, tol, max_iter=500)
    for solver, ref, key in ((gasa.GASA_SOLVER_CG, ref_cg, "pcg"),
                             (gasa.GASA_SOLVER_STATIONARY, ref_st, "stationary")):
        ctx, _ = gpu_setup(name, keep=False, solver=solver)
        try:
            x = np.zeros_like(pr.rhs)
            info = gasa.gasa_solve(ctx, pr.rhs, x, tol)
            assert info.converged and info.rel_residual <= tol
            assert abs(info.iterations - ref.iterations) <= 1, (solver, info.iterations, ref.iterations)
            assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-6
            paper = table[flux][key][M]
            if key == "pcg":
                assert abs(info.iterations - paper) <= 2, (name, info.iterations, paper)
            else:
                assert paper <= info.iterations <= paper + 4, (name, info.iterations, paper)
        finally:
            gasa.gasa_destroy(ctx)


def _real_index(sizes, s):
    """dof numbers of the real (unpadded) dofs of a level stored with s per unit"""
    return np.concatenate([i * s + np.arange(z) for i, z in enumerate(sizes)])


@pytest.mark.parametrize("dtail", DTAIL)
@pytest.mark.parametrize("name,hstar", [("p2_8", True), ("c1", True), ("uneq6", False)])
def test_padded_levels(name, hstar, dtail):
    """Unequal kept counts on a level, stored padded.  With the Section 4.3
    h*-step at the top every element is its own aggregate and keeps the
    singular vectors above 1e-3 sigma_1 (block sizes differ between units for
    p2_8); without it, aggregates of unequal size keep unequal h-branch
    counts (uneq6).  Kept counts bit-exact; unpadded A_k, w D^-1, P match the
    oracle; the padding holds zeros with 1 on A's diagonal; V-cycle, CG and
    served solves match."""
    gasa = _gasa()
    pr = problem(name)
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=pr.dim,
                hstar=hstar)
    ctx, info = gpu_setup(name, keep=True, hstar=1 if hstar else 0, dense_tail_dofs=dtail)
    tol = level_tolerances(H)
    try:
        assert info.n_levels == len(H.levels) == len(pr.agg_of) + 1 + (1 if hstar else 0)
        padded_seen = False
        for k, L in enumerate(H.levels):
            sh = gasa.gasa_level_shape(ctx, k)
            sizes = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_SIZES, np.zeros(sh["units"], np.int32))
            np.testing.assert_array_equal(sizes, np.diff(L.unit_ptr))
            assert sh["dofs"] == L.n == info.dofs[k]
            padded_seen |= bool(np.any(sizes != sh["s"]))
            idx = _real_index(sizes, sh["s"])
            rp, col, val = _level_bsr(gasa, ctx, k, "A", sh, sh["s"], sh["s"], sh["units"])
            Afull = bsr_scipy(rp, col, val)
            assert sparse_rel(Afull[idx][:, idx], L.A) <= tol[k]
            pad = np.setdiff1d(np.arange(sh["units"] * sh["s"]), idx)
            if pad.size:
                Ap = Afull[pad][:, pad].toarray()
                assert np.array_equal(Ap, np.eye(pad.size))
                assert abs(Afull[pad][:, idx]).max() == 0.0
            if k == len(H.levels) - 1:
                n_all = sh["units"] * sh["s"]
                Ci = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_COARSE_INV,
                                         np.zeros(n_all * n_all)).reshape(n_all, n_all)
                assert rel_err(Ci[np.ix_(idx, idx)], np.linalg.inv(H.coarse)) <= 100 * tol[k]
                continue
            assert abs(info.omega[k] - L.omega) <= 1e-2 * tol[k] * L.omega
            W = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_W,
                                    np.zeros(sh["units"] * sh["s"] ** 2)).reshape(-1, sh["s"], sh["s"])
            Wref = L.W.blocks if L.W.uniform else L.W.blocks
            for i in range(sh["units"]):
                z = sizes[i]
                assert rel_err(W[i, :z, :z], Wref[i]) <= tol[k]
            sn = sh["s_next"]
            n_next = H.levels[k + 1].unit_ptr.size - 1
            nsz = gasa.gasa_get_level(ctx, k + 1, gasa.GASA_LV_SIZES, np.zeros(n_next, np.int32))
            idx_n = _real_index(nsz, sn)
            prp, pcol, pval = _level_bsr(gasa, ctx, k, "P", sh, sh["s"], sn, sh["units"])
            Pg = bsr_scipy(prp, pcol, pval, n_next)
            assert sparse_rel(Pg[idx][:, idx_n], L.P) <= tol[k + 1]
            pad_n = np.setdiff1d(np.arange(n_next * sn), idx_n)
            if pad_n.size:
                assert abs(Pg[:, pad_n]).max() == 0.0
        if name in ("p2_8", "uneq6"):
            assert padded_seen
        want = O.make_vcycle(H)(pr.rhs)
        z = to_dev(np.zeros_like(pr.rhs))
        gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z)
        assert rel_err(to_host(z), want) <= 0.1 * tol[-1]
        ref = O.solve(H, pr.rhs, TOL, "cg", max_iter=5000)
        x = np.zeros_like(pr.rhs)
        inf = gasa.gasa_solve(ctx, pr.rhs, x, TOL)
        assert inf.converged and abs(inf.iterations - ref.iterations) <= 1
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= TOL
        ref32 = O.solve(H, pr.rhs, TOL, "cg", precision="mixed32", max_iter=5000)
        inf32 = gasa.gasa_solve(ctx, pr.rhs, x, TOL, gasa.GASA_PREC_MIXED32)
        assert inf32.converged and abs(inf32.iterations - ref32.iterations) <= 1
        srv = gasa.gasa_server_create(0, 8 << 30, 2)
        try:
            t = gasa.gasa_server_submit(srv, gasa.gasa_server_add_mesh(srv, ctx), pr.rhs, TOL)
            gasa.gasa_server_drain(srv, 300.0)
            xs = np.zeros_like(pr.rhs)
            st, si = gasa.gasa_server_poll(srv, t, xs)
            assert st == gasa.GASA_OK and abs(si.iterations - ref.iterations) <= 1
            assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= TOL
        finally:
            gasa.gasa_server_destroy(srv)
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("name", ["c1", "p3_32", "cd_q2_16", "tet_p2_6", "uneq6"])
def test_fused_tail(name):
    """The bottom levels and the coarsest solve run as one thread-block-cluster
    launch (tail_kib large) or as one launch per step (tail_kib = 0).  Both
    compute the V-cycle of Alg. 2 with the same sum per output row, so the
    two agree to rounding, both follow the oracle's V-cycle, and the solves
    they drive take the same number of iterations (+-1)."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    n_levels = len(H.levels)
    ctx_f, _ = gpu_setup(name, keep=False, tail_kib=1 << 20)
    ctx_s, _ = gpu_setup(name, keep=False, tail_kib=0, dense_tail_dofs=0)
    try:
        for prec, oprec, tol in ((gasa.GASA_PREC_FP64, "fp64", 1e-12),
                                 (gasa.GASA_PREC_MIXED32, "fp32", 1e-5)):
            # every level from 1 down qualifies by size; the tail starts lower
            # only where a CTA's share of the rows would overflow shared memory
            tf = gasa.gasa_tail_info(ctx_f, prec)
            assert 1 <= tf["first_level"] <= n_levels - 2 and tf["cluster"] in (8, 16), tf
            assert tf["coarse_inside"] == 1
            assert gasa.gasa_tail_info(ctx_s, prec) == {"first_level": n_levels - 1, "cluster": 0,
                                                        "coarse_inside": 0}
            want = O.make_vcycle(H, oprec)(pr.rhs)
            r = to_dev(pr.rhs)
            zf, zs = to_dev(np.zeros_like(pr.rhs)), to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_f, r, zf, prec)
            gasa.gasa_vcycle(ctx_s, r, zs, prec)
            zf, zs = to_host(zf), to_host(zs)
            assert rel_err(zf, zs) <= tol
            assert rel_err(zf, want) <= max(tol, 0.1 * level_tolerances(H)[-1])
            # a second call on the same buffers gives the same bits
            z2 = to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_f, r, z2, prec)
            assert np.array_equal(to_host(z2), zf)
        if pr.solver == "cg":
            for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32):
                xf, xs = np.zeros_like(pr.rhs), np.zeros_like(pr.rhs)
                inf_f = gasa.gasa_solve(ctx_f, pr.rhs, xf, TOL, prec)
                inf_s = gasa.gasa_solve(ctx_s, pr.rhs, xs, TOL, prec)
                assert inf_f.converged and inf_f.rel_residual <= TOL
                assert abs(inf_f.iterations - inf_s.iterations) <= 1
                assert np.linalg.norm(xf - xs) / np.linalg.norm(xs) <= 10 * TOL
    finally:
        gasa.gasa_destroy(ctx_f)
        gasa.gasa_destroy(ctx_s)


@pytest.mark.parametrize("name", ["c1", "p3_16", "p3_32", "uneq6", "tet_p2_6", "cd_q2_16"])
def test_grid_tail(name):
    """The coarse levels as one persistent cooperative launch (grid_tail = 1)
    against one launch per step: the range starts at the first level from
    which every level is unpadded with one block size s <= 8 (none for the
    P2 tets and the Q2 quads, whose coarse blocks are larger); where it runs,
    V-cycles agree with the per-step launches to rounding (1e-12 FP64,
    1e-5 FP32), follow the oracle's V-cycle, repeat bit for bit, and drive
    CG solves of the same iteration count (+-1)."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    n_levels = len(H.levels)
    sizes = [int(L.unit_ptr[1] - L.unit_ptr[0]) for L in H.levels]
    uniform = [all(np.all(np.diff(H.levels[j].unit_ptr) == sizes[k]) for j in range(k, n_levels))
               for k in range(n_levels)]
    expect = n_levels - 1
    for k in range(n_levels - 2, 0, -1):
        if sizes[k] <= 8 and all(sizes[j] == sizes[k] for j in range(k, n_levels)) and uniform[k]:
            expect = k
        else:
            break
    ctx_g, _ = gpu_setup(name, keep=False, grid_tail=1)
    ctx_s, _ = gpu_setup(name, keep=False, grid_tail=0, dense_tail_dofs=0)
    try:
        for prec, oprec, tol in ((gasa.GASA_PREC_FP64, "fp64", 1e-12),
                                 (gasa.GASA_PREC_MIXED32, "fp32", 1e-5)):
            tg = gasa.gasa_tail_info(ctx_g, prec)
            assert tg["first_level"] == expect, (tg, expect, sizes)
            if expect == n_levels - 1:
                assert tg == {"first_level": n_levels - 1, "cluster": 0, "coarse_inside": 0}
                continue
            assert tg["cluster"] > 0 and tg["cluster"] % 152 == 0 and tg["coarse_inside"] == 1
            want = O.make_vcycle(H, oprec)(pr.rhs)
            r = to_dev(pr.rhs)
            zg, zs = to_dev(np.zeros_like(pr.rhs)), to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_g, r, zg, prec)
            gasa.gasa_vcycle(ctx_s, r, zs, prec)
            zg, zs = to_host(zg), to_host(zs)
            assert rel_err(zg, zs) <= tol
            assert rel_err(zg, want) <= max(tol, 0.1 * level_tolerances(H)[-1])
            z2 = to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_g, r, z2, prec)
            assert np.array_equal(to_host(z2), zg)
        if pr.solver == "cg" and expect < n_levels - 1:
            for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32, gasa.GASA_PREC_MIXED16):
                xg, xs = np.zeros_like(pr.rhs), np.zeros_like(pr.rhs)
                inf_g = gasa.gasa_solve(ctx_g, pr.rhs, xg, TOL, prec)
                inf_s = gasa.gasa_solve(ctx_s, pr.rhs, xs, TOL, prec)
                assert inf_g.converged and inf_g.rel_residual <= TOL
                assert abs(inf_g.iterations - inf_s.iterations) <= 1
                assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) <= 10 * TOL
                # the graph-resident loop and the host-driven one agree bit for bit
                gasa.gasa_profile_enable(ctx_g, True)
                xh = np.zeros_like(pr.rhs)
                inf_h = gasa.gasa_solve(ctx_g, pr.rhs, xh, TOL, prec)
                gasa.gasa_profile_enable(ctx_g, False)
                assert inf_h.iterations == inf_g.iterations and np.array_equal(xh, xg)
    finally:
        gasa.gasa_destroy(ctx_g)
        gasa.gasa_destroy(ctx_s)


def test_grid_tail_wait_budget_runs_out():
    """With a 1 ns budget the persistent launch's grid barriers run out: the
    launch ends early and sets the error flag, gasa_vcycle and gasa_solve
    return GASA_ERR_TIMEOUT (the GPU stays usable), and the same context
    then solves normally once it is set up with the default budget."""
    gasa = _gasa()
    pr = problem("p3_16")
    ctx, _ = gpu_setup("p3_16", keep=False, grid_tail=1, wait_budget_s=1e-9)
    try:
        assert gasa.gasa_tail_info(ctx, gasa.GASA_PREC_MIXED32)["coarse_inside"] == 1
        r = to_dev(pr.rhs)
        z = to_dev(np.zeros_like(pr.rhs))
        for prec in (gasa.GASA_PREC_MIXED32, gasa.GASA_PREC_FP64):
            with pytest.raises(gasa.GasaError) as ei:
                gasa.gasa_vcycle(ctx, r, z, prec)
            assert ei.value.status == gasa.GASA_ERR_TIMEOUT
            x = np.zeros_like(pr.rhs)
            with pytest.raises(gasa.GasaError) as ei:
                gasa.gasa_solve(ctx, pr.rhs, x, TOL, prec)
            assert ei.value.status == gasa.GASA_ERR_TIMEOUT
    finally:
        gasa.gasa_destroy(ctx)
    ctx, _ = gpu_setup("p3_16", keep=False, grid_tail=1)
    try:
        x = np.zeros_like(pr.rhs)
        info = gasa.gasa_solve(ctx, pr.rhs, x, TOL, gasa.GASA_PREC_MIXED32)
        assert info.converged and info.rel_residual <= TOL
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.parametrize("name", ["c1", "p3_16", "p3_32", "tet_p2_4", "cd_q2_16", "uneq6"])
def test_fused_restriction(name):
    """Residual and restriction fused as b_{k+1} = R_k b_k - (R_k A_k) u_k
    (fused_restriction = 1, the default) against the two-step form
    R_k (b_k - A_k u_k) of Alg. 2 (fused_restriction = 0).  R_k A_k is kept
    exactly on the levels where it holds no more values than A_k; its block
    pattern is the structural pattern of R_k A_k (bit-exact) and its values
    follow the oracle's product; V-cycles agree with the two-step ones and the
    oracle's to rounding, and solves take the same iterations (+-1)."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    tol = level_tolerances(H)
    ctx_f, _ = gpu_setup(name, keep=False, fused_restriction=1, dense_tail_dofs=0)
    ctx_u, _ = gpu_setup(name, keep=False, fused_restriction=0, dense_tail_dofs=0)
    try:
        kept = 0
        for k, L in enumerate(H.levels[:-1]):
            RA = (L.R @ L.A).tocsr()
            units, n_next = L.unit_ptr.size - 1, H.levels[k + 1].unit_ptr.size - 1
            s, sn = int(np.max(np.diff(L.unit_ptr))), int(np.max(np.diff(H.levels[k + 1].unit_ptr)))
            pat = ((L.Ppat.T @ L.Apat) != 0).astype(np.float64).tocsr()
            optr, ocol = O.pattern_csr(pat)
            fits = ocol.size * s * sn <= L.Apat.nnz * s * s
            try:
                rp = gasa.gasa_get_level(ctx_f, k, gasa.GASA_LV_RA_ROWPTR, np.zeros(n_next + 1, np.int32))
            except gasa.GasaError:
                assert not fits, (k, "R A missing although it fits")
                continue
            assert fits, (k, "R A kept although larger than A")
            kept += 1
            np.testing.assert_array_equal(rp, optr)
            col = gasa.gasa_get_level(ctx_f, k, gasa.GASA_LV_RA_COL, np.zeros(rp[-1], np.int32))
            np.testing.assert_array_equal(col, ocol)
            if np.all(np.diff(L.unit_ptr) == s) and np.all(np.diff(H.levels[k + 1].unit_ptr) == sn):
                val = gasa.gasa_get_level(ctx_f, k, gasa.GASA_LV_RA_VAL,
                                          np.zeros(rp[-1] * sn * s)).reshape(-1, sn, s)
                G = bsr_scipy(rp, col, val, units)
                # entries of R_k within tol[k+1] max|R_k| and of A_k within
                # tol[k] max|A_k| perturb an entry of R_k A_k by at most
                # tol[k+1] max|R_k| ||A_k||_1 + tol[k] max|A_k| ||R_k||_inf
                # (the cancellation in R_k A_k, smooth rows against A_k, keeps
                # max|R_k A_k| well below both)
                bound = (tol[k + 1] * abs(L.R).max() * np.asarray(abs(L.A).sum(axis=0)).max()
                         + tol[k] * abs(L.A).max() * np.asarray(abs(L.R).sum(axis=1)).max())
                assert sparse_rel(G, RA) <= bound / abs(RA).max()
        assert kept >= 1
        for prec, oprec, tl in ((gasa.GASA_PREC_FP64, "fp64", 1e-11),
                                (gasa.GASA_PREC_MIXED32, "fp32", 1e-5),
                                (gasa.GASA_PREC_MIXED16, "fp16", 1e-5)):
            want = O.make_vcycle(H, oprec)(pr.rhs)
            r = to_dev(pr.rhs)
            zf, zu = to_dev(np.zeros_like(pr.rhs)), to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_f, r, zf, prec)
            gasa.gasa_vcycle(ctx_u, r, zu, prec)
            zf, zu = to_host(zf), to_host(zu)
            assert rel_err(zf, zu) <= tl, (oprec, rel_err(zf, zu))
            assert rel_err(zf, want) <= (max(tl, 0.1 * tol[-1]) if oprec == "fp64" else 1e-4)
        solver = gasa.GASA_SOLVER_CG if pr.solver == "cg" else gasa.GASA_SOLVER_GMRES
        if solver == gasa.GASA_SOLVER_CG:
            for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32):
                xf, xu = np.zeros_like(pr.rhs), np.zeros_like(pr.rhs)
                inf_f = gasa.gasa_solve(ctx_f, pr.rhs, xf, TOL, prec)
                inf_u = gasa.gasa_solve(ctx_u, pr.rhs, xu, TOL, prec)
                assert inf_f.converged and inf_f.rel_residual <= TOL
                assert abs(inf_f.iterations - inf_u.iterations) <= 1
    finally:
        gasa.gasa_destroy(ctx_f)
        gasa.gasa_destroy(ctx_u)


@pytest.mark.parametrize("name", ["c1", "p3_16", "p3_32", "cd_q2_16", "tet_p2_6", "uneq6"])
def test_dense_tail(name):
    """The bottom of the V-cycle as one dense operator (dense_tail_dofs, on by
    default).  From the first level k >= 1 whose levels down to N - 1 hold at
    most dense_tail_dofs stored dofs, Alg. 2 from u_k = 0 is the linear map
    b_k -> u_k; setup forms it by running those steps on the unit vectors.  The
    stored operator matches the oracle's V-cycle of the sub-hierarchy k .. N
    applied to the unit vectors; V-cycles agree with the per-step ones
    (dense_tail_dofs = 0) to rounding and with the oracle's; solves take the
    same iterations (+-1)."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    tol = level_tolerances(H)
    N = len(H.levels) - 1
    thr = gasa.gasa_default_options().dense_tail_dofs
    ctx_d, _ = gpu_setup(name, keep=False)
    ctx_s, _ = gpu_setup(name, keep=False, dense_tail_dofs=0)
    try:
        ci = gasa.gasa_cycle_info(ctx_s)
        assert (ci["dense_first_level"], ci["dense_n"]) == (N, 0)
        stored = [gasa.gasa_level_shape(ctx_d, k) for k in range(N + 1)]
        want_k = N
        for k in range(N - 1, 0, -1):
            if stored[k]["units"] * stored[k]["s"] > thr:
                break
            want_k = k
        info = gasa.gasa_cycle_info(ctx_d)
        assert want_k < N, "every workload here has a small bottom"
        assert info["dense_first_level"] == want_k
        kt = want_k
        n = stored[kt]["units"] * stored[kt]["s"]
        assert info["dense_n"] == n
        with pytest.raises(gasa.GasaError):
            gasa.gasa_get_level(ctx_s, kt, gasa.GASA_LV_DENSE_TAIL, np.zeros(n * n))
        M = gasa.gasa_get_level(ctx_d, kt, gasa.GASA_LV_DENSE_TAIL, np.zeros(n * n)).reshape(n, n)
        sizes = gasa.gasa_get_level(ctx_d, kt, gasa.GASA_LV_SIZES,
                                    np.zeros(stored[kt]["units"], np.int32))
        idx = _real_index(sizes, stored[kt]["s"])
        sub = O.Hierarchy(levels=H.levels[kt:], coarse=H.coarse, t_pre=H.t_pre, t_post=H.t_post)
        V = O.make_vcycle(sub)
        nr = idx.size
        Mref = np.column_stack([V(np.eye(nr)[:, j]) for j in range(nr)])
        assert rel_err(M[np.ix_(idx, idx)], Mref) <= 0.1 * tol[-1]
        pad = np.setdiff1d(np.arange(n), idx)
        if pad.size:
            # padding entries of b never reach real entries of u
            assert np.max(np.abs(M[np.ix_(idx, pad)])) == 0.0
            assert np.max(np.abs(M[np.ix_(pad, idx)])) == 0.0
        for prec, oprec, tl in ((gasa.GASA_PREC_FP64, "fp64", 1e-11),
                                (gasa.GASA_PREC_MIXED32, "fp32", 1e-5),
                                (gasa.GASA_PREC_MIXED16, "fp16", 1e-5)):
            want = O.make_vcycle(H, oprec)(pr.rhs)
            r = to_dev(pr.rhs)
            zd, zs = to_dev(np.zeros_like(pr.rhs)), to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_d, r, zd, prec)
            gasa.gasa_vcycle(ctx_s, r, zs, prec)
            zd, zs = to_host(zd), to_host(zs)
            assert rel_err(zd, zs) <= tl, (oprec, rel_err(zd, zs))
            assert rel_err(zd, want) <= (max(tl, 0.1 * tol[-1]) if oprec == "fp64" else 1e-4)
        solver = gasa.GASA_SOLVER_CG if pr.solver == "cg" else gasa.GASA_SOLVER_GMRES
        for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32):
            xd, xs = np.zeros_like(pr.rhs), np.zeros_like(pr.rhs)
            inf_d = gasa.gasa_solve(ctx_d, pr.rhs, xd, TOL, prec)
            inf_s = gasa.gasa_solve(ctx_s, pr.rhs, xs, TOL, prec)
            assert inf_d.converged and inf_d.rel_residual <= TOL
            assert abs(inf_d.iterations - inf_s.iterations) <= 1
            assert np.linalg.norm(xd - xs) / np.linalg.norm(xs) <= 10 * TOL
    finally:
        gasa.gasa_destroy(ctx_d)
        gasa.gasa_destroy(ctx_s)


def test_dense_tail_option_range():
    """dense_tail_dofs outside 0 .. 8192 is rejected by setup."""
    gasa = _gasa()
    for bad in (-1, 8193):
        with pytest.raises(gasa.GasaError) as ei:
            gpu_setup("tiny", keep=False, dense_tail_dofs=bad)
        assert ei.value.status == gasa.GASA_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["c1", "p3_16", "tet_p2_4", "cd_q2_16", "hex_M3"])
def test_folded_smoother(name):
    """Level 0 smoothing in the folded form u + c - (w D^-1 A) u with
    c = w D^-1 b (folded_smoother, on by default) against the plain step
    u + w D^-1 (b - A u) of Alg. 1 (folded_smoother = 0).  The stored
    w D_0^-1 A_0 follows the oracle's product W_0 A_0 in A_0's pattern; V-cycles
    agree with the plain ones to rounding (bit for bit with FP16 level-0
    blocks, which keep the plain step) and with the oracle's; solves take the
    same iterations (+-1); the host-driven loop's per-launch byte count of a
    level-0 step is that of W A, c, u and the result."""
    gasa = _gasa()
    H = oracle_setup(name)
    pr = problem(name)
    tol = level_tolerances(H)
    ctx_f, _ = gpu_setup(name, keep=True)
    ctx_u, _ = gpu_setup(name, keep=True, folded_smoother=0)
    try:
        assert gasa.gasa_cycle_info(ctx_f)["folded"] == 1
        assert gasa.gasa_cycle_info(ctx_u)["folded"] == 0
        sh = gasa.gasa_level_shape(ctx_f, 0)
        s, n, nnzb = sh["s"], sh["units"], sh["nnzb"]
        with pytest.raises(gasa.GasaError):
            gasa.gasa_get_level(ctx_u, 0, gasa.GASA_LV_WA, np.zeros(nnzb * s * s))
        rp, col, _ = _level_bsr(gasa, ctx_f, 0, "A", sh, s, s, n)
        wa = gasa.gasa_get_level(ctx_f, 0, gasa.GASA_LV_WA, np.zeros(nnzb * s * s)).reshape(-1, s, s)
        G = bsr_scipy(rp, col, wa)
        L0 = H.levels[0]
        Wm = L0.W.to_sparse()
        ref = (Wm @ L0.A).tocsr()
        # W_0 within tol[0] max|W_0| and A_0 within tol[0] max|A_0| perturb an
        # entry of W_0 A_0 by at most tol[0] (max|W| ||A||_1 + max|A| ||W||_inf)
        bound = tol[0] * (abs(Wm).max() * np.asarray(abs(L0.A).sum(axis=0)).max()
                          + abs(L0.A).max() * np.asarray(abs(Wm).sum(axis=1)).max())
        assert sparse_rel(G, ref) <= bound / abs(ref).max()
        # FP64 and the FP16-block level 0 keep the plain step: same bits
        for prec, oprec, tl in ((gasa.GASA_PREC_FP64, "fp64", 0.0),
                                (gasa.GASA_PREC_MIXED32, "fp32", 1e-5),
                                (gasa.GASA_PREC_MIXED16, "fp16", 0.0)):
            want = O.make_vcycle(H, oprec)(pr.rhs)
            r = to_dev(pr.rhs)
            zf, zu = to_dev(np.zeros_like(pr.rhs)), to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx_f, r, zf, prec)
            gasa.gasa_vcycle(ctx_u, r, zu, prec)
            zf, zu = to_host(zf), to_host(zu)
            if tl == 0.0:
                assert np.array_equal(zf, zu)
            else:
                assert rel_err(zf, zu) <= tl, (oprec, rel_err(zf, zu))
            assert rel_err(zf, want) <= (0.1 * tol[-1] if oprec == "fp64" else 1e-4)
        solver = gasa.GASA_SOLVER_CG if pr.solver == "cg" else gasa.GASA_SOLVER_GMRES
        for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32):
            xf, xu = np.zeros_like(pr.rhs), np.zeros_like(pr.rhs)
            inf_f = gasa.gasa_solve(ctx_f, pr.rhs, xf, TOL, prec)
            inf_u = gasa.gasa_solve(ctx_u, pr.rhs, xu, TOL, prec)
            assert inf_f.converged and inf_f.rel_residual <= TOL
            assert abs(inf_f.iterations - inf_u.iterations) <= 1
        if solver == gasa.GASA_SOLVER_CG:
            gasa.gasa_profile_enable(ctx_f, True)
            x = np.zeros_like(pr.rhs)
            gasa.gasa_solve(ctx_f, pr.rhs, x, TOL, gasa.GASA_PREC_MIXED32)
            _, launches, by = gasa.gasa_profile_read(ctx_f, 0)
            gasa.gasa_profile_enable(ctx_f, False)
            assert launches > 0
            want_bytes = nnzb * s * s * 4 + 4 * nnzb + 4 * (n + 1) + 3 * n * s * 4
            assert by / launches == want_bytes
    finally:
        gasa.gasa_destroy(ctx_f)
        gasa.gasa_destroy(ctx_u)


@pytest.mark.parametrize("tpre,tpost", [(0, 2), (1, 1), (2, 0)])
@pytest.mark.parametrize("name", ["c1", "p3_16"])
def test_smoothing_counts(name, tpre, tpost):
    """Alg. 2 with other pre/post smoothing counts than Section 6's 3 and 3,
    including none on one side: the V-cycle (folded level-0 steps, dense
    bottom operator and fused restriction at their defaults) follows the
    oracle's with the same counts."""
    import dataclasses
    gasa = _gasa()
    H = dataclasses.replace(oracle_setup(name), t_pre=tpre, t_post=tpost)
    pr = problem(name)
    ctx, _ = gpu_setup(name, keep=False, t_pre=tpre, t_post=tpost)
    try:
        for prec, oprec in ((gasa.GASA_PREC_FP64, "fp64"), (gasa.GASA_PREC_MIXED32, "fp32")):
            want = O.make_vcycle(H, oprec)(pr.rhs)
            z = to_dev(np.zeros_like(pr.rhs))
            gasa.gasa_vcycle(ctx, to_dev(pr.rhs), z, prec)
            tl = 0.1 * level_tolerances(H)[-1] if oprec == "fp64" else 1e-4
            assert rel_err(to_host(z), want) <= tl, (oprec, rel_err(to_host(z), want))
    finally:
        gasa.gasa_destroy(ctx)
