"""Pins of the CPU oracle against what the paper and the mathematics fix:
closed forms, invariants and brute force on tiny inputs.  Each pin is
chosen so that a plausible slip (a dropped term, a flipped sign, a wrong
index or a transposed operand) in the oracle fails it."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp

from oracle import gasa_oracle as O
from synth import configs, random_ops as RO

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CONST = json.load(open(os.path.join(GOLD, "paper_constants.json")))
SIZES = json.load(open(os.path.join(GOLD, "hierarchy_sizes.json")))


def lap1d(n):
    return sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], (n, n)).tocsr()


def lap1d_modes(n):
    """eigenpairs of tridiag(-1, 2, -1)/2 (= D^{-1} A for 1x1 blocks)"""
    k = np.arange(1, n + 1)
    lam = 1.0 - np.cos(k * np.pi / (n + 1))
    i = np.arange(1, n + 1)
    V = np.sin(np.outer(i, k) * np.pi / (n + 1)) * np.sqrt(2.0 / (n + 1))
    return lam, V


def scalar_blocks(A):
    return O.BlockDiag(np.arange(A.shape[0] + 1), A.diagonal().reshape(-1, 1, 1))


@pytest.fixture(scope="module")
def tiny():
    pr = configs.poisson2d(8, 1, r=12, n_levels=3, name="tiny")
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)
    return pr, H


@pytest.fixture(scope="module")
def tiny2level():
    pr = configs.poisson2d(8, 1, r=12, n_levels=2, name="tiny2")
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)
    return pr, H


# ---------------------------------------------------------------------------
def test_splitmix_published_outputs():
    g = CONST["splitmix64_seed0"]["value"]
    u = O.splitmix_uniform(0, 0, 3)
    want = np.array([int(h, 16) >> 11 for h in g], dtype=np.float64) * 2.0 ** -53
    np.testing.assert_array_equal(u, want)


def test_library_defaults_are_the_papers():
    from paper_2504_13373_gb300 import gasa
    try:
        opt = gasa.gasa_default_options()
    except RuntimeError:
        pytest.skip("libgasa.so not built")
    assert opt.gamma == CONST["gamma"]["value"]
    assert opt.q_power == CONST["q_power"]["value"]
    assert opt.omega_factor == CONST["omega_factor"]["value"]
    assert opt.t_pre == CONST["t_pre"]["value"] and opt.t_post == CONST["t_post"]["value"]


def test_block_inverse_identity():
    pr = configs.poisson2d_p1()
    S = pr.A.to_scipy()
    D = O.block_diagonal(S, np.arange(pr.A.n + 1) * 3)
    Dinv = O.invert_blocks(D)
    err = np.max(np.abs(np.einsum("uij,ujk->uik", D.blocks, Dinv.blocks) - np.eye(3)))
    assert err <= 1e-12
    # D really is the block diagonal: D = A on diagonal blocks, A - D has none
    R = (S - D.to_sparse()).tocsr()
    for u in range(0, pr.A.n, 97):
        assert np.max(np.abs(R[3 * u:3 * u + 3, 3 * u:3 * u + 3].toarray())) == 0.0


def test_power_estimate_closed_form():
    """1-D Laplacian, 1x1 blocks: D^{-1} A has eigenpairs (lam_k, v_k).  From
    x0 = (v_1 + v_n)/sqrt(2), q steps give x ~ lam_1^q v_1 + lam_n^q v_n and
    the estimate sqrt(lam_1^{2q+2} + lam_n^{2q+2}) / sqrt(lam_1^{2q} + lam_n^{2q})."""
    n, q = 50, 3
    A = lap1d(n)
    lam, V = lap1d_modes(n)
    x0 = (V[:, 0] + V[:, -1]) / np.sqrt(2.0)
    got = O.power_estimate(A, O.invert_blocks(scalar_blocks(A)), x0, q)
    a, b = lam[0], lam[-1]
    want = np.sqrt(a ** (2 * q + 2) + b ** (2 * q + 2)) / np.sqrt(a ** (2 * q) + b ** (2 * q))
    assert abs(got - want) <= 1e-12 * want


def test_power_estimate_below_spectral_radius(tiny):
    pr, H = tiny
    L = H.levels[0]
    ev = np.linalg.eigvals(L.Dinv.to_sparse().toarray() @ L.A.toarray())
    rho = np.max(np.abs(ev))
    assert L.rho <= rho * (1 + 1e-12)
    assert L.rho >= 0.5 * rho
    assert abs(L.omega - CONST["omega_factor"]["value"] / L.rho) <= 1e-15 * L.omega


def test_relax_closed_form_two_modes():
    """x0 = a v_1 + b v_n: after m sweeps x = a mu_1^m v_1 + b mu_n^m v_n with
    mu = 1 - w lam; the stop sweep is the first m where
    ||x^(m-1)|| / ||x^(m)|| < 1 + gamma."""
    n, w, gamma = 40, 0.8, 0.03
    A = lap1d(n)
    lam, V = lap1d_modes(n)
    W = O.invert_blocks(scalar_blocks(A)).scaled(w)
    a, b = 1.0, 50.0
    x0 = a * V[:, 0] + b * V[:, -1]
    mu1, mun = 1 - w * lam[0], 1 - w * lam[-1]
    nrm = lambda m: np.hypot(a * mu1 ** m, b * mun ** m)
    m_stop = next(m for m in range(1, 1000) if nrm(m - 1) / nrm(m) < 1 + gamma)
    Bx, sw = O.relax_candidates(A, W, x0[:, None], gamma, 1000)
    assert sw[0] == m_stop
    want = a * mu1 ** m_stop * V[:, 0] + b * mun ** m_stop * V[:, -1]
    assert np.max(np.abs(Bx[:, 0] - want)) <= 1e-12 * np.max(np.abs(want))


def test_relax_cap_and_identity_smoother():
    """D^{-1}A = I (diagonal A), w = 4/3: x <- x - (4/3) x = -x/3, the norm
    ratio is always 3 so the cap stops it; after m sweeps x = (-1/3)^m x0."""
    n = 10
    A = sp.diags(np.arange(1.0, n + 1)).tocsr()
    W = O.invert_blocks(scalar_blocks(A)).scaled(4.0 / 3.0)
    x0 = RO.random_vector(n, 3)
    Bx, sw = O.relax_candidates(A, W, x0[:, None], 0.03, 7)
    assert sw[0] == 7
    np.testing.assert_allclose(Bx[:, 0], (-1.0 / 3.0) ** 7 * x0, rtol=1e-14)


@pytest.mark.parametrize("rows,r,ncut,want", [
    (12, 12, 3, 4), (40, 4, 3, 4), (16, 12, 3, 5), (20, 12, 3, 6), (80, 80, 6, 13),
    (104, 80, 6, 17), (176, 80, 6, 29), (5, 12, 8, 1), (2, 12, 3, 1), (3, 2, 1, 2)])
def test_keep_count_rule(rows, r, ncut, want):
    """Eq. sik h-branch: |A_j| / n_cut floored, at least one, at most r and rows."""
    assert O.keep_count(rows, r, ncut) == want


def test_default_cut_factor():
    assert 2 ** 2 - (2 - 1) == CONST["n_cut_2d"]["value"]
    assert 2 ** 3 - (3 - 1) == CONST["n_cut_3d"]["value"]


def test_level_sizes_workload_p1():
    pr = configs.poisson2d_p1()
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)
    assert [L.n for L in H.levels] == SIZES["poisson2d_p1_32x32"]["dofs"]
    assert O.median_aggregate_dofs(pr.agg_of[0], H.levels[0].unit_ptr, 512) == 12


@pytest.mark.parametrize("name,units,fan,b,r,ncut", [
    ("poisson3d_p2_48cubed", 663552, 8, 10, 80, 6),
    ("poisson2d_p3_256x256", 131072, 4, 10, 4, 3)])
def test_level_sizes_structure(name, units, fan, b, r, ncut):
    want = SIZES[name]["dofs"]
    dofs, s, n = [units * b], b, units
    while len(dofs) < len(want):
        s = O.keep_count(fan * s, r, ncut)
        n //= fan
        dofs.append(n * s)
    assert dofs == want


def test_tentative_isometry_and_sign(tiny):
    pr, H = tiny
    for L in H.levels[:-1]:
        T = L.T.toarray()
        assert np.max(np.abs(T.T @ T - np.eye(T.shape[1]))) <= 1e-13
        for c in range(T.shape[1]):
            m = np.argmax(np.abs(T[:, c]))
            assert T[m, c] > 0


def test_tentative_reproduces_candidates_full_rank():
    """s_j >= rank(B_j): T_j T_j^T B_j = B_j (the isometry spans the
    candidates, Eq. splitB)."""
    n_units, bs, r = 64, 10, 4
    B = np.asfortranarray(RO.random_normal(n_units * bs * r, 9).reshape(r, -1).T)
    agg = RO.chunk_aggregates(n_units, 4)
    T, ptr, _ = O.tentative(B, agg, np.arange(n_units + 1) * bs, 16, 3.0)
    assert np.all(np.diff(ptr) == 4)
    assert np.max(np.abs(T @ (T.T @ B) - B)) <= 1e-13 * np.max(np.abs(B))


def test_tentative_eckart_young():
    """Truncation keeps the dominant singular directions:
    ||B_j - T_j T_j^T B_j||_F^2 = sum of the discarded sigma_l^2."""
    n_units, bs, r = 32, 3, 12
    B = np.asfortranarray(RO.random_normal(n_units * bs * r, 10).reshape(r, -1).T)
    agg = RO.chunk_aggregates(n_units, 4)
    up = np.arange(n_units + 1) * bs
    T, ptr, sv = O.tentative(B, agg, up, 8, 3.0)
    rows = O.aggregate_rows(agg, up, 8)
    for J in range(8):
        BJ = B[rows[J], :]
        TJ = T[rows[J], ptr[J]:ptr[J + 1]].toarray()
        resid = np.linalg.norm(BJ - TJ @ (TJ.T @ BJ)) ** 2
        s = ptr[J + 1] - ptr[J]
        assert abs(resid - np.sum(sv[J][s:] ** 2)) <= 1e-10 * np.sum(sv[J] ** 2)
        # the discarded part is the smallest: any other s-subspace does worse
        Q, _ = np.linalg.qr(BJ[:, :s])
        assert resid <= np.linalg.norm(BJ - Q @ (Q.T @ BJ)) ** 2 + 1e-12


def test_smoothed_prolongator_lowers_energy(tiny):
    """P = (I - w D^{-1} A) T with w rho(D^{-1}A) < 2 lowers the A-energy of
    every column (Eq. TR0 smoothing step); a wrong sign raises it."""
    pr, H = tiny
    L = H.levels[0]
    A = L.A.toarray()
    P, T = L.P.toarray(), L.T.toarray()
    eP = np.einsum("ic,ij,jc->c", P, A, P)
    eT = np.einsum("ic,ij,jc->c", T, A, T)
    assert np.all(eP < eT)
    assert np.all(P[np.abs(T) > 0] != 0.0)
    # one smoothing step spreads each column of T by one ring of A's pattern
    # and no further
    reach = (np.abs(A) @ np.abs(T)) > 0
    assert np.all((P != 0.0) <= (reach | (T != 0.0)))


def test_restriction_is_transpose_and_galerkin_projection(tiny):
    """R = P^T exactly, and P A_c^{-1} P^T A is an A-self-adjoint projection
    iff A_c = P^T A P (Galerkin)."""
    pr, H = tiny
    for k, L in enumerate(H.levels[:-1]):
        assert (L.R - L.P.T).count_nonzero() == 0
        A, P = L.A.toarray(), L.P.toarray()
        Ac = H.levels[k + 1].A.toarray()
        Pi = P @ np.linalg.solve(Ac, P.T @ A)
        assert np.max(np.abs(Pi @ Pi - Pi)) <= 1e-10
        assert np.max(np.abs(A @ Pi - (A @ Pi).T)) <= 1e-10 * np.max(np.abs(A))


def test_coarse_operators_spd(tiny):
    pr, H = tiny
    for L in H.levels:
        Ad = L.A.toarray()
        assert np.max(np.abs(Ad - Ad.T)) <= 1e-12 * np.max(np.abs(Ad))
        la.cholesky(0.5 * (Ad + Ad.T))


def test_patterns_structural(tiny):
    """P's block pattern = pattern(A) x aggregation; A_{k+1} pattern covers
    every stored block of R A P."""
    pr, H = tiny
    for k, L in enumerate(H.levels[:-1]):
        agg = np.asarray(pr.agg_of[k])
        Ap = L.Apat.tocsr()
        for i in range(Ap.shape[0]):
            want = sorted({int(agg[j]) for j in Ap.indices[Ap.indptr[i]:Ap.indptr[i + 1]]})
            got = sorted(L.Ppat.indices[L.Ppat.indptr[i]:L.Ppat.indptr[i + 1]].tolist())
            assert got == want


def test_two_grid_error_operator(tiny2level):
    """Two levels: I - M A = S^t_post (I - P A_c^{-1} R A) S^t_pre with
    S = I - W A (the textbook error propagation of Alg. 2)."""
    pr, H = tiny2level
    L = H.levels[0]
    n = L.n
    M = O.make_vcycle(H)
    Mm = np.column_stack([M(e) for e in np.eye(n)])
    A = L.A.toarray()
    W = L.W.to_sparse().toarray()
    S = np.eye(n) - W @ A
    P, R = L.P.toarray(), L.R.toarray()
    C = np.eye(n) - P @ np.linalg.solve(H.coarse, R @ A)
    E = np.linalg.matrix_power(S, H.t_post) @ C @ np.linalg.matrix_power(S, H.t_pre)
    assert np.max(np.abs((np.eye(n) - Mm @ A) - E)) <= 1e-10


def test_vcycle_linear_symmetric_convergent(tiny):
    pr, H = tiny
    M = O.make_vcycle(H)
    r1 = RO.random_vector(pr.n_dofs, 1)
    r2 = RO.random_vector(pr.n_dofs, 2)
    z = M(2.5 * r1 + r2)
    assert np.max(np.abs(z - (2.5 * M(r1) + M(r2)))) <= 1e-12 * np.max(np.abs(z))
    assert abs(M(r1) @ r2 - r1 @ M(r2)) <= 1e-11 * abs(M(r1) @ r2)
    n = pr.n_dofs
    Mm = np.column_stack([M(e) for e in np.eye(n)])
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(n) - Mm @ H.levels[0].A.toarray())))
    assert rho < 1.0


def test_vcycle_bottom_is_a_fixed_linear_map(tiny):
    """Alg. 2 below level k, started from u_k = 0, is a fixed linear map of b_k:
    a two-level cycle on level 0 whose coarse solve applies the sub-hierarchy's
    V-cycle (levels 1 .. N) as a matrix M_1, formed from its action on the unit
    vectors, is the full V-cycle (the dense bottom operator of the library).
    A cycle that used the level-1 operator's inverse instead, or skipped the
    level-1 smoothing, would differ."""
    pr, H = tiny
    assert H.N >= 2
    sub = O.Hierarchy(levels=H.levels[1:], coarse=H.coarse, t_pre=H.t_pre, t_post=H.t_post)
    V1 = O.make_vcycle(sub)
    n1 = H.levels[1].n
    M1 = np.column_stack([V1(e) for e in np.eye(n1)])
    two = O.Hierarchy(levels=H.levels[:2], coarse=np.linalg.inv(M1), t_pre=H.t_pre,
                      t_post=H.t_post)
    full, split = O.make_vcycle(H), O.make_vcycle(two)
    f = RO.random_vector(pr.n_dofs, 5)
    zf, zs = full(f), split(f)
    assert np.max(np.abs(zs - zf)) <= 1e-10 * np.max(np.abs(zf))
    # the exact level-1 solve in its place gives a different (two-grid) cycle
    exact = O.Hierarchy(levels=H.levels[:2], coarse=H.levels[1].A.toarray(), t_pre=H.t_pre,
                        t_post=H.t_post)
    assert np.max(np.abs(O.make_vcycle(exact)(f) - zf)) > 1e-6 * np.max(np.abs(zf))


def test_pcg_matches_direct_solve(tiny):
    pr, H = tiny
    res = O.solve(H, pr.rhs, 1e-12)
    x = np.linalg.solve(H.levels[0].A.toarray(), pr.rhs)
    assert res.converged
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)


@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_iterates_minimise_the_energy_error(flexible):
    """With SPD A and a fixed SPD preconditioner M, the k-th PCG iterate is
    the point of K_k(M A, M b) nearest to x* in the A-norm (brute force: an
    orthonormal basis of the explicit powers and the Galerkin system), for
    k = 1..6, whether beta is the plain or the Polak-Ribiere one (they agree
    for a fixed M).  A slip in alpha, the residual update or beta fails it."""
    rng = np.random.default_rng(12)
    n = 40
    B = rng.standard_normal((n, n))
    A = B @ B.T / n + 0.5 * np.eye(n)
    C = rng.standard_normal((n, n))
    Mm = np.diag(1.0 / np.diag(A)) + 0.01 * (C @ C.T) / n
    b = rng.standard_normal(n)
    for k in range(1, 7):
        got = O.pcg(sp.csr_matrix(A), b, lambda r: Mm @ r, 1e-300, k, flexible=flexible).x
        K = [Mm @ b]
        for _ in range(k - 1):
            K.append(Mm @ (A @ K[-1]))
        Q, _ = np.linalg.qr(np.column_stack(K))
        want = Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want), k


def test_cg_finite_termination():
    """CG (M = I) on a matrix with k distinct eigenvalues converges in k steps."""
    lam = np.repeat([1.0, 3.0, 7.0, 20.0], 25)
    A = sp.diags(lam).tocsr()
    b = RO.random_vector(lam.size, 4)
    res = O.pcg(A, b, lambda r: r.copy(), 1e-10, 50)
    assert res.converged and res.iterations <= 4


def test_gmres_finite_termination_and_direct():
    """GMRES (M = I) on a diagonalizable nonsymmetric matrix with k distinct
    eigenvalues needs at most k steps; with a V-cycle it matches a direct solve."""
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((60, 60))
    Dg = np.diag(np.repeat([1.0, 2.0, 5.0], 20))
    A = sp.csr_matrix(Q @ Dg @ np.linalg.inv(Q))
    b = RO.random_vector(60, 5)
    res = O.gmres(A, b, lambda r: r.copy(), 1e-10, restart=30, max_iter=10)
    assert res.converged and res.iterations <= 3
    x = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(res.x - x) <= 1e-8 * np.linalg.norm(x)


def _min_residual_iterate(A, Mm, b, x0, k, right):
    """Brute force: the iterate of k steps of minimal residual from x0 over the
    Krylov space, built from explicit powers and orthonormalised by QR, with
    the least-squares problem solved by lstsq.  Left preconditioning
    minimises ||M (b - A x)|| over x0 + K_k(M A, M r0); right preconditioning
    minimises ||b - A x|| over x0 + M K_k(A M, r0)."""
    r0 = b - A @ x0
    start, op = (r0, A @ Mm) if right else (Mm @ r0, Mm @ A)
    K = [start]
    for _ in range(k - 1):
        K.append(op @ K[-1])
    Q, _ = np.linalg.qr(np.column_stack(K))
    c = np.linalg.lstsq(op @ Q, start, rcond=None)[0]
    return x0 + (Mm @ (Q @ c) if right else Q @ c)


@pytest.mark.parametrize("flexible", [False, True])
def test_gmres_iterates_are_minimal_residual(flexible):
    """Each GMRES iterate minimises the (left-preconditioned, or with
    `flexible` the true) residual over its Krylov space, checked against a
    brute-force least-squares solve for k = 1..6 steps, and a restart begins a
    new minimisation from the last iterate (GMRES(3), two cycles).  A slip in
    the Arnoldi orthogonalisation, the Givens rotations or the update of x
    fails it."""
    rng = np.random.default_rng(11)
    n = 40
    A = 3.0 * np.eye(n) + 0.4 * rng.standard_normal((n, n)) + np.triu(0.3 * rng.standard_normal((n, n)), 1)
    Mm = np.diag(1.0 / np.diag(A)) + 0.02 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    As = sp.csr_matrix(A)

    def M(r):
        return Mm @ r

    for k in range(1, 7):
        got = O.gmres(As, b, M, 1e-300, restart=30, max_iter=k, flexible=flexible).x
        want = _min_residual_iterate(A, Mm, b, np.zeros(n), k, flexible)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want), k
    got = O.gmres(As, b, M, 1e-300, restart=3, max_iter=6, flexible=flexible).x
    x3 = _min_residual_iterate(A, Mm, b, np.zeros(n), 3, flexible)
    want = _min_residual_iterate(A, Mm, b, x3, 3, flexible)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_gmres_and_fcg_on_workload(tiny):
    pr, H = tiny
    x = np.linalg.solve(H.levels[0].A.toarray(), pr.rhs)
    for kw in [dict(solver="gmres"), dict(solver="cg", precision="mixed32"),
               dict(solver="gmres", precision="mixed32")]:
        res = O.solve(H, pr.rhs, 1e-10, **kw)
        assert res.converged and res.rel_residual <= 1e-10
        assert np.linalg.norm(res.x - x) <= 1e-7 * np.linalg.norm(x)


def test_candidate_transfer_tt_option(tiny):
    """Eq. SA_Bk: with B^{k+1} = T^T B^k and s_j >= rank, T B^{k+1} = B^k."""
    pr = configs.poisson2d(8, 3, r=4, n_levels=3, name="tiny_p3")
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=4, dim=2, cand_init="T")
    L0, L1 = H.levels[0], H.levels[1]
    assert np.max(np.abs(L0.T @ L1.B_in - L0.B)) <= 1e-12 * np.max(np.abs(L0.B))


def test_stationary_solver(tiny):
    pr, H = tiny
    res = O.stationary(H, pr.rhs, 1e-8, 400)
    assert res.converged


def test_stationary_error_contracts_by_the_iteration_operator(tiny):
    """Alg. 2 as a stationary solver from x = 0: the error e_k = x* - x_k is
    e_k = E^k x* with E = I - M A, M the V-cycle as a matrix.  E is
    self-adjoint in the A inner product (symmetric cycle), so every step
    shrinks ||e||_A by at most ||E||_A = rho(E) (a dense eigenvalue problem,
    computed apart from the solver), and the ratio of successive A-norm errors
    tends to rho(E).  An update that dropped x, flipped the correction's sign or
    corrected with b instead of the residual fails the first bound."""
    pr, H = tiny
    A = H.levels[0].A.toarray()
    n = A.shape[0]
    M = O.make_vcycle(H)
    Mm = np.column_stack([M(e) for e in np.eye(n)])
    L = np.linalg.cholesky(A)
    Et = L.T @ (np.eye(n) - Mm @ A) @ np.linalg.inv(L.T)      # E in the A inner product
    assert np.max(np.abs(Et - Et.T)) <= 1e-10
    rho = np.max(np.abs(np.linalg.eigvalsh(0.5 * (Et + Et.T))))
    assert 0.0 < rho < 1.0
    xs = np.linalg.solve(A, pr.rhs)
    errs = [np.sqrt(xs @ A @ xs)]
    for k in range(1, 26):
        e = xs - O.stationary(H, pr.rhs, 1e-300, k).x
        errs.append(np.sqrt(e @ A @ e))
    for k in range(25):
        assert errs[k + 1] <= rho * errs[k] * (1 + 1e-8) + 1e-13 * errs[0], k
    late = (errs[25] / errs[20]) ** (1 / 5)
    assert 0.9 * rho <= late <= rho * (1 + 1e-8), (late, rho)


@pytest.mark.parametrize("seed,n_agg", [(1, 7), (2, 8), (3, 1), (4, 2)])
def test_median_aggregate_dofs_is_the_lower_median(seed, n_agg):
    """Section 4.2's r: the median dof count of the level-1 aggregates, the
    lower one for an even count (statistics.median_low), on aggregates of
    unequal sizes built from units of unequal dof counts."""
    import statistics
    rng = np.random.default_rng(seed)
    n_units = 3 * n_agg + 2
    dofs = rng.integers(1, 12, n_units)
    unit_ptr = np.concatenate([[0], np.cumsum(dofs)])
    agg = np.concatenate([np.arange(n_agg), rng.integers(0, n_agg, n_units - n_agg)])
    rng.shuffle(agg)
    sizes = [int(sum(dofs[u] for u in range(n_units) if agg[u] == a)) for a in range(n_agg)]
    assert O.median_aggregate_dofs(agg, unit_ptr, n_agg) == statistics.median_low(sizes)


def test_fp16_block_storage():
    """Values k/1024 of the block maximum are stored exactly; otherwise the
    dequantised value is within half an FP16 unit (2^-11 relative to the
    block maximum) of the original, and zero blocks stay zero."""
    s = 3.5
    exact = np.array([[[1.0, -0.5, 0.25], [3.0 / 1024, 0.0, -1.0]]]) * s
    np.testing.assert_array_equal(O.fp16_blocks(exact), exact.astype(np.float32))
    blocks = RO.random_blocks(200, 5, 81) * np.exp(RO.random_vector(200, 82) * 5)[:, None, None]
    blocks[7] = 0.0
    d = O.fp16_blocks(blocks)
    m = np.max(np.abs(blocks), axis=(1, 2))
    err = np.max(np.abs(d - blocks), axis=(1, 2))
    assert np.all(err <= 2.0 ** -11 * m * (1 + 1e-6) + 1e-300)
    assert np.all(d[7] == 0.0)


def test_null_singular_vectors_completed_deterministically():
    """A rank-1 block (every candidate column a multiple of e_0) keeping two
    vectors: the first is e_0, the second (zero singular value) is the
    Gram-Schmidt completion of e_1 against e_0, i.e. e_1."""
    rows, r = 4, 3
    B = np.zeros((rows, r))
    B[0, :] = [2.0, -1.0, 0.5]
    T, ptr, sv = O.tentative(B, np.zeros(1, dtype=np.int64), np.array([0, rows]), 1, 1.0, keep=[2])
    Td = T.toarray()
    np.testing.assert_allclose(Td[:, 0], [1, 0, 0, 0], atol=1e-15)
    np.testing.assert_allclose(Td[:, 1], [0, 1, 0, 0], atol=1e-15)
    # rank 2 with s = 3: the completion is orthogonal to the two real vectors
    B = RO.random_normal(6 * 2, 3).reshape(6, 2) @ RO.random_normal(2 * 5, 4).reshape(2, 5)
    T, _, sv = O.tentative(B, np.zeros(1, dtype=np.int64), np.array([0, 6]), 1, 1.0, keep=[3])
    Td = T.toarray()
    assert sv[0][2] <= 1e-10 * sv[0][0]
    assert np.max(np.abs(Td.T @ Td - np.eye(3))) <= 1e-14
    assert np.max(np.abs(Td[:, :2] @ (Td[:, :2].T @ B) - B)) <= 1e-12 * np.max(np.abs(B))


def test_matrix_free_levels_apply_the_galerkin_operator():
    """Section 4.4: A_k applied as R_{k-1} A_{k-1} P_{k-1} equals the stored
    Galerkin operator (to rounding), at every matrix-free depth, and a V-cycle
    with matrix-free levels is the same preconditioner."""
    pr = configs.poisson2d(8, 1, r=12, n_levels=4, name="tiny4")
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)
    assert H.N == 3
    rng = np.random.default_rng(7)
    prev = H.levels[0].A
    for k in range(1, H.N):
        prev = O.GalerkinOperator(H.levels[k - 1].R, prev, H.levels[k - 1].P)
        x = rng.standard_normal(H.levels[k].A.shape[0])
        ref = H.levels[k].A @ x
        assert np.linalg.norm(prev @ x - ref) <= 1e-12 * np.linalg.norm(ref)
    f = rng.standard_normal(H.levels[0].A.shape[0])
    u0 = O.make_vcycle(H)(f)
    for kappa in range(1, H.N):
        u = O.make_vcycle(H, matrix_free_levels=kappa)(f)
        assert np.linalg.norm(u - u0) <= 1e-11 * np.linalg.norm(u0)
    # with kappa = 0 nothing changes, bit for bit
    assert np.array_equal(O.make_vcycle(H, matrix_free_levels=0)(f), u0)


def test_hstar_keep_rule():
    """Eq. sik, h*-branch: keep the singular values above delta sigma_1."""
    U, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((10, 4)))
    V, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((6, 4)))
    for sv, want in (([1.0, 0.5, 1e-4, 1e-9], 2), ([1.0, 0.9, 0.8, 0.7], 4), ([2.0, 1e-5, 0, 0], 1)):
        B = U @ np.diag(sv) @ V.T
        S = np.linalg.svd(B, compute_uv=False)
        assert O.hstar_keep(S, 1e-3) == want


def test_hstar_top_level():
    """Section 4.3: with an h*-step the first coarse level has one unit per
    element, each keeping the singular vectors above 1e-3 sigma_1 of its own
    candidate rows (so the level-1 block sizes vary), T is an isometry, the
    remaining levels follow the given aggregates, and the preconditioned CG
    still converges."""
    pr = configs.poisson2d(8, 2, r=24, n_levels=3, name="tiny_p2")
    H = O.setup(pr.A.row_ptr, pr.A.col, pr.A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2, hstar=True)
    assert len(H.levels) == len(pr.agg_of) + 2
    L0, L1 = H.levels[0], H.levels[1]
    assert L1.unit_ptr.size == L0.unit_ptr.size
    sizes = np.diff(L1.unit_ptr)
    for J, S in enumerate(L0.svals):
        assert sizes[J] == O.hstar_keep(S, 1e-3)
    assert sizes.max() <= pr.A.b and sizes.min() >= 1
    TT = (L0.T.T @ L0.T).toarray()
    assert np.abs(TT - np.eye(TT.shape[0])).max() <= 1e-12
    assert H.levels[2].unit_ptr.size - 1 == int(pr.agg_of[0].max()) + 1
    res = O.solve(H, pr.rhs, 1e-10, "cg", max_iter=500)
    assert res.converged


def test_flexible_cg_beta_three_steps_exact():
    """Flexible CG (Polak-Ribiere beta_k = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k)
    worked by hand in exact rational arithmetic on a 3x3 SPD system whose
    preconditioner changes between calls (diag(1, 1/2, 1/3), then the
    identity, then the diagonal again).  The first beta equals the plain
    r1.z1 / r0.z0 (r1 is orthogonal to p0 = z0); the second does not, so a
    slip between the two forms fails here.  The oracle's third iterate must
    equal the exact one to rounding."""
    from fractions import Fraction as F
    A = [[F(4), F(1), F(0)], [F(1), F(3), F(1)], [F(0), F(1), F(2)]]
    b = [F(1), F(2), F(3)]
    diag = [F(1), F(1, 2), F(1, 3)]
    precs = [lambda r: [d * v for d, v in zip(diag, r)], lambda r: r[:],
             lambda r: [d * v for d, v in zip(diag, r)]]

    def mv(M, v):
        return [sum(M[i][j] * v[j] for j in range(3)) for i in range(3)]

    def dot(u, v):
        return sum(x * y for x, y in zip(u, v))

    x = [F(0)] * 3
    r = b[:]
    z = precs[0](r)
    p = z[:]
    betas = []
    for k in range(3):
        q = mv(A, p)
        alpha = dot(r, z) / dot(p, q)
        x = [xi + alpha * pi for xi, pi in zip(x, p)]
        r_new = [ri - alpha * qi for ri, qi in zip(r, q)]
        if k == 2:
            break
        z_new = precs[k + 1](r_new)
        beta = dot(r_new, [u - v for u, v in zip(z_new, z)]) / dot(r, z)
        betas.append((beta, dot(r_new, z_new) / dot(r, z)))
        p = [zi + beta * pi for zi, pi in zip(z_new, p)]
        r, z = r_new, z_new
    assert betas[0][0] == betas[0][1] and betas[1][0] != betas[1][1]

    diag_f = np.array([1.0, 0.5, 1.0 / 3.0])
    calls = []

    def M(v):
        calls.append(1)
        return v * diag_f if len(calls) != 2 else v.copy()

    Ad = np.array([[float(v) for v in row] for row in A])
    bd = np.array([float(v) for v in b])
    want = np.array([float(v) for v in x])
    res = O.pcg(sp.csr_matrix(Ad), bd, M, tol=1e-300, max_iter=3, flexible=True)
    assert np.max(np.abs(res.x - want)) <= 1e-14 * np.max(np.abs(want))
    calls.clear()
    plain = O.pcg(sp.csr_matrix(Ad), bd, M, tol=1e-300, max_iter=3, flexible=False)
    assert np.max(np.abs(plain.x - want)) > 1e-8 * np.max(np.abs(want))


@pytest.mark.parametrize("p,r,ns,growth", [(1, 12, (16, 32, 64), 1.6), (3, 4, (16, 32), 2.05)])
def test_2d_count_growth_under_refinement_is_bounded(p, r, ns, growth):
    """The 2-D SIPG workloads' CG counts (penalty 10 p^2 / h) grow under
    refinement, for the reasons the convergence study gives (block Jacobi
    does not damp continuous grid-scale modes at this penalty multiple, and
    with r = 4 the coarse space holds one vector per element); the growth per
    halving of h stays within the bound measured when it was explained
    (P1, r = 12: 18 / 27 / 41; P3, r = 4: 232 / 444), so a change that makes
    the method converge worse fails here."""
    from synth import configs
    counts = []
    for n in ns:
        pr = configs.poisson2d(n, p, r=r)
        A = pr.A
        H = O.setup(A.row_ptr, A.col, A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)
        res = O.solve(H, pr.rhs, 1e-10, "cg", max_iter=2000)
        assert res.converged
        counts.append(res.iterations)
    for a, b_ in zip(counts[:-1], counts[1:]):
        assert b_ <= growth * a, counts
