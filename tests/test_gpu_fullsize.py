"""Full-size parity on the benchmark workload (P3 SIPG, 256x256, 1.31M dofs)
in the launch configuration bench.py times, plus full-size solve properties
of the 3-D P2 and convection-diffusion workloads.

The oracle finishes the whole level-0 setup of the benchmark workload in
seconds (block inverses, Alg. 4, Eq. bsmooth, per-aggregate SVD, P, R and
the Galerkin product), so level 0 is compared element by element; the
oracle's full solve would take about an hour, so the solves are checked by
properties that hold at any size: the true residual recomputed on the host
(scipy) is at most 1e-10, mixed and FP64 counts agree within +-1, and a
second solve repeats the first bit for bit.
"""
import functools

import numpy as np
import pytest

from oracle import gasa_oracle as O
from synth import configs
from tests.helpers import bsr_scipy, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _gasa():
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    return gasa


@functools.lru_cache(maxsize=None)
def _bench_problem():
    return configs.poisson2d_p3()


def _setup(gasa, pr, keep=True, solver=0):
    A = pr.A
    ctx = gasa.gasa_create(0)
    opt = gasa.gasa_default_options(dim=pr.dim, n_cand=pr.r, keep_setup_data=1 if keep else 0,
                                    solver=solver, max_iter=20000)
    info = gasa.gasa_setup(ctx, A.row_ptr, A.col, A.val.ravel(), A.b, pr.agg_of, opt,
                           adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx, centroids=pr.centroids,
                           init_candidates=pr.B0)
    return ctx, info


@functools.lru_cache(maxsize=None)
def _bench_oracle():
    pr = _bench_problem()
    A = pr.A
    return O.setup(A.row_ptr, A.col, A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)


def _sparse_rel(G, Ref):
    D = (G - Ref).tocsr()
    return (np.max(np.abs(D.data)) if D.nnz else 0.0) / np.max(np.abs(Ref.data))


def test_benchmark_workload_level0_setup_matches_oracle():
    gasa = _gasa()
    pr = _bench_problem()
    A = pr.A
    S = A.to_scipy()
    up = np.arange(A.n + 1) * A.b
    # oracle, level 0 of Alg. 5, step by step
    Dinv = O.invert_blocks(O.block_diagonal(S, up))
    rho = O.power_estimate(S, Dinv, O.power_start_vector(configs.SEED, 0, S.shape[0]), 3)
    omega = O.omega_from_rho(rho)
    W = Dinv.scaled(omega)
    B, sweeps = O.relax_candidates(S, W, pr.B0[:, :pr.r], 0.03, 100)
    agg = np.asarray(pr.agg_of[0], np.int64)
    n1 = int(agg.max()) + 1
    T, _, svals = O.tentative(B, agg, up, n1, 3.0)
    P = O.smoothed_prolongator(S, W, T)
    A1 = O.galerkin(P.T.tocsr(), S, P)
    ctx, info = _setup(gasa, pr)
    try:
        assert abs(info.rho[0] - rho) <= 1e-12 * rho
        assert abs(info.omega[0] - omega) <= 1e-12 * omega
        sh = gasa.gasa_level_shape(ctx, 0)
        sw = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_SWEEPS, np.zeros(pr.r, np.int32))
        np.testing.assert_array_equal(sw, sweeps)
        Wg = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_W, np.zeros(A.n * A.b * A.b))
        assert rel_err(Wg, W.blocks.ravel()) <= 1e-12
        Bg = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_CAND, np.zeros(A.n * A.b * pr.r))
        assert rel_err(Bg.reshape(pr.r, -1).T, B) <= 1e-11
        gap = min((sv[3] - sv[4]) / sv[0] if sv.size > 4 else sv[3] / sv[0] for sv in svals)
        tolT = max(1e-10, 100 * 2.2e-16 / gap)
        Tg = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_T_VAL, np.zeros(A.n * A.b * 4)).reshape(A.n * A.b, 4)
        Tref = np.zeros_like(Tg)
        Tc = T.tocsr()
        for J in range(n1):
            rows = np.nonzero(np.repeat(agg == J, A.b))[0]
            Tref[rows] = Tc[rows][:, 4 * J:4 * J + 4].toarray()
        assert np.max(np.abs(Tg - Tref)) <= tolT
        n_p = sh["P_nnzb"]
        prp = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_P_ROWPTR, np.zeros(A.n + 1, np.int32))
        pcol = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_P_COL, np.zeros(n_p, np.int32))
        pval = gasa.gasa_get_level(ctx, 0, gasa.GASA_LV_P_VAL, np.zeros(n_p * 40)).reshape(n_p, 10, 4)
        Pg = bsr_scipy(prp, pcol, pval, n1)
        assert _sparse_rel(Pg, P) <= max(1e-10, tolT)
        sh1 = gasa.gasa_level_shape(ctx, 1)
        arp = gasa.gasa_get_level(ctx, 1, gasa.GASA_LV_A_ROWPTR, np.zeros(n1 + 1, np.int32))
        acol = gasa.gasa_get_level(ctx, 1, gasa.GASA_LV_A_COL, np.zeros(sh1["nnzb"], np.int32))
        aval = gasa.gasa_get_level(ctx, 1, gasa.GASA_LV_A_VAL, np.zeros(sh1["nnzb"] * 16)).reshape(-1, 4, 4)
        A1g = bsr_scipy(arp, acol, aval)
        # bit-exact structural block patterns of P and A_1
        Apat = O.bool_csr(A.row_ptr.astype(np.int64), A.col.astype(np.int64), (A.n, A.n))
        Ppat = ((Apat @ O.aggregation_matrix(agg, n1)) != 0).astype(np.float64).tocsr()
        A1pat = ((Ppat.T @ ((Apat @ Ppat) != 0).astype(np.float64)) != 0).astype(np.float64)
        optr, ocol = O.pattern_csr(Ppat)
        np.testing.assert_array_equal(prp, optr)
        np.testing.assert_array_equal(pcol, ocol)
        optr, ocol = O.pattern_csr(A1pat)
        np.testing.assert_array_equal(arp, optr)
        np.testing.assert_array_equal(acol, ocol)
        assert _sparse_rel(A1g, A1) <= max(1e-10, tolT)
    finally:
        gasa.gasa_destroy(ctx)


def _solve_properties(gasa, pr, solver, expect_iters=None):
    ctx, info = _setup(gasa, pr, keep=False, solver=solver)
    S = pr.A.to_scipy()
    bn = np.linalg.norm(pr.rhs)
    try:
        res = {}
        for prec in (gasa.GASA_PREC_MIXED32, gasa.GASA_PREC_FP64):
            x = np.zeros_like(pr.rhs)
            si = gasa.gasa_solve(ctx, pr.rhs, x, TOL, prec)
            assert si.converged
            assert np.linalg.norm(pr.rhs - S @ x) / bn <= TOL
            res[prec] = (si.iterations, x)
        assert abs(res[gasa.GASA_PREC_MIXED32][0] - res[gasa.GASA_PREC_FP64][0]) <= 1
        x2 = np.zeros_like(pr.rhs)
        si2 = gasa.gasa_solve(ctx, pr.rhs, x2, TOL, gasa.GASA_PREC_MIXED32)
        assert si2.iterations == res[gasa.GASA_PREC_MIXED32][0]
        assert np.array_equal(x2, res[gasa.GASA_PREC_MIXED32][1])
        return info, res
    finally:
        gasa.gasa_destroy(ctx)


def test_benchmark_workload_solves():
    gasa = _gasa()
    pr = _bench_problem()
    info, res = _solve_properties(gasa, pr, gasa.GASA_SOLVER_CG)
    assert [info.dofs[k] for k in range(info.n_levels)] == \
        [1310720, 131072, 32768, 8192, 2048, 512, 128, 32, 8]


@pytest.mark.slow
def test_poisson3d_p2_full_size_solves():
    """48^3 x 6 Kuhn tets, SIPG P2 (6.64M dofs), r = 80, L0..L4."""
    gasa = _gasa()
    pr = configs.poisson3d_p2()
    info, res = _solve_properties(gasa, pr, gasa.GASA_SOLVER_CG)
    assert [info.dofs[k] for k in range(info.n_levels)] == [6635520, 1078272, 176256, 28512, 4698]


@pytest.mark.slow
def test_convdiff_q2_full_size_solves():
    """512^2 jittered quads, LDG + upwind Q2 (2.36M dofs), GMRES(30), Pe = 100."""
    gasa = _gasa()
    pr = configs.convdiff2d_q2(peclet=100.0)
    info, res = _solve_properties(gasa, pr, gasa.GASA_SOLVER_GMRES)
    assert info.dofs[0] == 2359296


@pytest.mark.slow
@pytest.mark.parametrize("grid_tail", [0, 1])
def test_benchmark_workload_vcycle_matches_oracle(grid_tail):
    """One V-cycle of the full benchmark workload (9 levels) in FP64, FP32 and
    FP16-block precision, element by element against the oracle's V-cycle
    (Alg. 2) built from the oracle's own hierarchy, with the kernels the
    benchmark launches (thread-per-row level 0, lane-team coarse levels, or
    the persistent coarse launch).  Bars as for the small workloads: FP64
    within the hierarchy tolerance, FP32 and FP16 within 1e-4 of the
    oracle's emulation, FP16 within 1e-2 of FP64."""
    from tests.test_gpu_solver import level_tolerances
    gasa = _gasa()
    pr = _bench_problem()
    H = _bench_oracle()
    A = pr.A
    ctx = gasa.gasa_create(0)
    try:
        opt = gasa.gasa_default_options(dim=2, n_cand=pr.r, keep_setup_data=0, max_iter=20000,
                                        grid_tail=grid_tail)
        gasa.gasa_setup(ctx, A.row_ptr, A.col, A.val.ravel(), A.b, pr.agg_of, opt,
                        adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx, centroids=pr.centroids,
                        init_candidates=pr.B0)
        assert (gasa.gasa_tail_info(ctx, gasa.GASA_PREC_MIXED32)["first_level"] == 1) == bool(grid_tail)
        import torch
        r = torch.from_numpy(pr.rhs).cuda()
        z = torch.zeros_like(r)
        want = O.make_vcycle(H, "fp64")(pr.rhs)
        gasa.gasa_vcycle(ctx, r, z, gasa.GASA_PREC_FP64)
        assert rel_err(z.cpu().numpy(), want) <= 0.1 * level_tolerances(H)[-1]
        wantf = O.make_vcycle(H, "fp32")(pr.rhs)
        gasa.gasa_vcycle(ctx, r, z, gasa.GASA_PREC_MIXED32)
        zf = z.cpu().numpy()
        assert rel_err(zf, wantf) <= 1e-4 and rel_err(zf, want) <= 1e-4
        wanth = O.make_vcycle(H, "fp16")(pr.rhs)
        gasa.gasa_vcycle(ctx, r, z, gasa.GASA_PREC_MIXED16)
        zh = z.cpu().numpy()
        assert rel_err(zh, wanth) <= 1e-4 and rel_err(zh, want) <= 1e-2
    finally:
        gasa.gasa_destroy(ctx)


@pytest.mark.slow
def test_benchmark_workload_solves_match_the_oracle_record():
    """The full benchmark solves against the oracle's own solves of the same
    workload (tests/golden/c2_oracle_solve.json, written by
    make_c2_oracle_solve.py: about an hour of oracle time per precision).
    Iteration counts within 1 of the oracle's (FP64 against FP64, mixed
    against mixed), and each solution within 1e-10 relative of the oracle's
    FP64 solution over the record's 4,096 sampled dofs (a sample estimate of
    ||x - x_oracle|| / ||x_oracle||; the oracle's own FP64 and mixed solutions
    differ by 3.7e-11)."""
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c2_oracle_solve.json")))
    gasa = _gasa()
    pr = _bench_problem()
    assert rec["dofs"] == pr.n_dofs
    idx = np.asarray(rec["sample_index"], dtype=np.int64)
    xo = np.asarray(rec["fp64"]["x_sample"])
    ctx, info = _setup(gasa, pr, keep=False)
    try:
        assert [info.dofs[k] for k in range(info.n_levels)] == rec["level_dofs"]
        for prec, key in ((gasa.GASA_PREC_FP64, "fp64"), (gasa.GASA_PREC_MIXED32, "mixed32")):
            x = np.zeros_like(pr.rhs)
            si = gasa.gasa_solve(ctx, pr.rhs, x, TOL, prec)
            assert si.converged and si.rel_residual <= TOL
            assert abs(si.iterations - rec[key]["iterations"]) <= 1, (key, si.iterations)
            err = np.linalg.norm(x[idx] - xo) / np.linalg.norm(xo)
            assert err <= TOL, (key, err)
    finally:
        gasa.gasa_destroy(ctx)
