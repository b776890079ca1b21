"""Single-operation parity: each CUDA kernel behind the C ABI against the CPU
oracle on the same seeded inputs.

Tolerances: FP64 kernels change only the summation order of <= a few
hundred products per entry, so entries agree to 1e-12 relative to the
largest entry (a rounding-error bound of n * eps * cond with n <= 10^3 and
cond <= 10^3 leaves a wide margin).  FP32 kernels are compared with the FP64
oracle at 2e-5 (n * 2^-24 for n <= 300 terms of unit-sized products).
"""
import numpy as np
import pytest

from oracle import gasa_oracle as O
from synth import random_ops as RO
from tests.helpers import bsr_scipy, problem, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def _gasa():
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    return gasa


CASES_MV = [
    # (n_rows, n_cols, br, bc, per_row, seed)
    (1031, 1031, 3, 3, 4, 1),     # ragged tail, vector width 1
    (517, 517, 10, 10, 4, 2),     # P3 triangles block, 16-byte vectors
    (300, 83, 10, 4, 3, 3),       # prolongator-shaped
    (83, 300, 4, 10, 9, 4),       # restriction-shaped
    (97, 61, 13, 17, 5, 5),       # wider than the templated sizes (generic path)
    (1, 1, 1, 1, 1, 6),           # smallest
    # long rows (>= 12 blocks on average): one warp per block row
    (203, 150, 4, 4, 20, 7),
    (100, 300, 5, 10, 24, 8),
    (64, 64, 36, 36, 16, 9),      # 36-row blocks: two rows per lane
    (50, 40, 13, 17, 30, 10),
    (33, 900, 4, 10, 70, 11),     # restriction-shaped, more blocks than lanes
    (70, 70, 8, 8, 20, 12),       # lane groups of 8
    (40, 40, 16, 16, 12, 13),     # lane groups of 16
    (20, 20, 32, 32, 8, 14),      # one lane group
    # (the cases above with <= 4096 block rows take one CTA per block row)
    (5000, 5000, 4, 4, 6, 21),    # > 4096 short-ish rows, few threads: lane groups of a warp
    (5000, 3000, 5, 10, 6, 22),   # same, non-power-of-two height: lane per block
    (4500, 4500, 13, 13, 5, 23),
    # square blocks of 2..8 with >= 6 blocks per row: a lane per block, teams
    # of 8, 32 or 128 lanes per block row by the average row length
    (2000, 2000, 2, 2, 10, 31),
    (300, 300, 3, 3, 60, 32),
    (257, 257, 5, 5, 140, 33),
    (129, 129, 7, 7, 30, 34),
    (1000, 997, 6, 6, 8, 35),
]


@pytest.mark.parametrize("case", CASES_MV)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_bsr_mv_fp64(case, mode):
    gasa = _gasa()
    n, m, br, bc, per, seed = case
    ptr, col, val = RO.random_bsr(n, m, br, bc, per, seed)
    x = RO.random_vector(m * bc, seed)
    b = RO.random_vector(n * br, seed, stream=120)
    y0 = RO.random_vector(n * br, seed, stream=121)
    Ax = bsr_scipy(ptr, col, val, m) @ x
    want = {0: Ax, 1: b - Ax, 2: y0 + Ax}[mode]
    y = to_dev(y0)
    gasa.gasa_bsr_mv(mode, n, br, bc, to_dev(ptr), to_dev(col), to_dev(val.ravel()), to_dev(x),
                     to_dev(b), y)
    assert rel_err(to_host(y), want) <= TOL64


@pytest.mark.parametrize("case", CASES_MV[:5] + CASES_MV[6:9] + CASES_MV[11:12] + CASES_MV[-5:])
def test_bsr_mv_fp32(case):
    gasa = _gasa()
    n, m, br, bc, per, seed = case
    ptr, col, val = RO.random_bsr(n, m, br, bc, per, seed)
    x = RO.random_vector(m * bc, seed)
    b = RO.random_vector(n * br, seed, stream=120)
    want = b - bsr_scipy(ptr, col, val, m) @ x
    y = to_dev(np.zeros(n * br, np.float32))
    gasa.gasa_bsr_mv_f32(1, n, br, bc, to_dev(ptr), to_dev(col), to_dev(val.ravel().astype(np.float32)),
                         to_dev(x.astype(np.float32)), to_dev(b.astype(np.float32)), y)
    assert rel_err(to_host(y), want) <= TOL32


def _split(v):
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


@pytest.mark.parametrize("case", CASES_MV[:6] + CASES_MV[6:9])
def test_bsr_mv_double_single(case):
    """Double-single product from exact FP32 splits of A and x: every entry
    within 2^-40 of sum |a x| of the FP64 product.  The splits hold a and x to
    2^-48 and the dropped lo * lo terms are below that; the FP32 low word takes
    one rounding of at most 2^-24 of its own size (a few 2^-24 of sum |a x|)
    per term, so n terms stay below n * 2^-47 of sum |a x| (n <= 700 here)."""
    gasa = _gasa()
    n, m, br, bc, per, seed = case
    ptr, col, val = RO.random_bsr(n, m, br, bc, per, seed)
    x = RO.random_vector(m * bc, seed)
    S = bsr_scipy(ptr, col, val, m)
    want = S @ x
    bound = 2.0 ** -40 * (abs(S) @ np.abs(x)) + 1e-300
    ah, al = _split(val.ravel())
    xh, xl = _split(x)
    y = to_dev(np.zeros(n * br))
    gasa.gasa_bsr_mv_ds(n, br, bc, to_dev(ptr), to_dev(col), to_dev(ah), to_dev(al), to_dev(xh),
                        to_dev(xl), y)
    got = to_host(y)
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)
    # the FP32 product alone misses that bound by orders of magnitude
    y32 = to_dev(np.zeros(n * br, np.float32))
    gasa.gasa_bsr_mv_f32(0, n, br, bc, to_dev(ptr), to_dev(col), to_dev(ah), to_dev(xh), None, y32)
    assert np.max(np.abs(to_host(y32) - want) / bound) > 100


def test_bsr_mv_workload_matrix():
    """The 32x32 P1 and 32x32 P3 SIPG operators, residual mode."""
    gasa = _gasa()
    for name in ("c1", "p3_32"):
        A = problem(name).A
        x = RO.random_vector(A.n * A.b, 7)
        b = RO.random_vector(A.n * A.b, 8)
        want = b - A.to_scipy() @ x
        y = to_dev(np.zeros_like(b))
        gasa.gasa_bsr_mv(1, A.n, A.b, A.b, to_dev(A.row_ptr), to_dev(A.col), to_dev(A.val.ravel()),
                         to_dev(x), to_dev(b), y)
        assert rel_err(to_host(y), want) <= TOL64


def _jacobi_inputs(n, bs, seed, per_row=4):
    ptr, col, val = RO.random_bsr(n, n, bs, bs, per_row, seed, diag=True)
    val = RO.diagonally_dominant(ptr, col, val)
    W = RO.random_blocks(n, bs, seed)
    x = RO.random_vector(n * bs, seed)
    b = RO.random_vector(n * bs, seed, stream=130)
    return ptr, col, val, W, x, b


@pytest.mark.parametrize("n,bs,seed,per_row", [
    (1031, 3, 11, 4), (517, 10, 12, 4), (129, 17, 13, 4), (77, 40, 14, 4),
    (301, 4, 15, 20), (97, 13, 16, 40), (40, 36, 17, 30),   # warp per block row
    (90, 8, 18, 16), (33, 16, 19, 12), (20, 32, 20, 8),     # CTA per block row
    (5000, 4, 24, 6), (4500, 13, 25, 5),                    # warp per block row
    (2000, 2, 36, 10), (300, 3, 37, 60), (257, 5, 38, 140),  # lane per block
    (129, 7, 39, 30), (1000, 6, 40, 8), (3001, 4, 41, 13)])
def test_jacobi_sweep_fp64(n, bs, seed, per_row):
    gasa = _gasa()
    ptr, col, val, W, x, b = _jacobi_inputs(n, bs, seed, per_row)
    A = bsr_scipy(ptr, col, val)
    Wd = O.BlockDiag(np.arange(n + 1) * bs, W)
    want = O.smooth_step(x, A, Wd, b)
    want_first = Wd.apply(b)
    out = to_dev(np.zeros(n * bs))
    dW, dval = to_dev(W.ravel()), to_dev(val.ravel())
    gasa.gasa_jacobi_sweep(n, bs, to_dev(ptr), to_dev(col), dval, dW, to_dev(x), to_dev(b), out)
    assert rel_err(to_host(out), want) <= TOL64
    gasa.gasa_jacobi_sweep(n, bs, to_dev(ptr), to_dev(col), dval, dW, None, to_dev(b), out, first=True)
    assert rel_err(to_host(out), want_first) <= TOL64


@pytest.mark.parametrize("n,bs,seed,per_row", [(1031, 3, 11, 4), (517, 10, 12, 4), (129, 17, 13, 4),
                                               (301, 4, 15, 20), (300, 3, 37, 60), (3001, 4, 41, 13),
                                               (129, 8, 42, 70)])
def test_jacobi_sweep_fp32(n, bs, seed, per_row):
    gasa = _gasa()
    ptr, col, val, W, x, b = _jacobi_inputs(n, bs, seed, per_row)
    A = bsr_scipy(ptr, col, val)
    want = O.smooth_step(x, A, O.BlockDiag(np.arange(n + 1) * bs, W), b)
    out = to_dev(np.zeros(n * bs, np.float32))
    f = np.float32
    gasa.gasa_jacobi_sweep_f32(n, bs, to_dev(ptr), to_dev(col), to_dev(val.ravel().astype(f)),
                               to_dev(W.ravel().astype(f)), to_dev(x.astype(f)), to_dev(b.astype(f)), out)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(to_host(out) - want)) / scale <= 1e-4


@pytest.mark.parametrize("name", ["c1", "p3_32", "tet_p2_4"])
def test_block_inverse(name):
    gasa = _gasa()
    A = problem(name).A
    up = np.arange(A.n + 1) * A.b
    D = O.block_diagonal(A.to_scipy(), up)
    want = 0.75 * O.invert_blocks(D).blocks
    W = to_dev(np.zeros(A.n * A.b * A.b))
    ns = gasa.gasa_block_inverse(A.n, A.b, to_dev(A.row_ptr), to_dev(A.col), to_dev(A.val.ravel()),
                                 0.75, W)
    assert ns == 0
    assert rel_err(to_host(W), want.ravel()) <= 1e-11


def test_block_inverse_singular_block_reported():
    gasa = _gasa()
    ptr, col, val = RO.random_bsr(64, 64, 4, 4, 3, 21, diag=True)
    val = RO.diagonally_dominant(ptr, col, val)
    k = int(np.nonzero(col[ptr[5]:ptr[6]] == 5)[0][0]) + ptr[5]
    val[k] = 0.0                                  # unit 5: zero diagonal block
    W = to_dev(np.zeros(64 * 16))
    ns = gasa.gasa_block_inverse(64, 4, to_dev(ptr), to_dev(col), to_dev(val.ravel()), 1.0, W)
    assert ns == 1


@pytest.mark.parametrize("name", ["c1", "p3_32"])
def test_power_estimate(name):
    gasa = _gasa()
    A = problem(name).A
    up = np.arange(A.n + 1) * A.b
    Dinv = O.invert_blocks(O.block_diagonal(A.to_scipy(), up))
    x0 = RO.random_vector(A.n * A.b, 31)
    want = O.power_estimate(A.to_scipy(), Dinv, x0 / np.linalg.norm(x0), 3)
    got = gasa.gasa_power_estimate(A.n, A.b, to_dev(A.row_ptr), to_dev(A.col), to_dev(A.val.ravel()),
                                   to_dev(Dinv.blocks.ravel()), to_dev(x0), 3)
    assert abs(got - want) <= 1e-12 * want


@pytest.mark.parametrize("name,r", [("c1", 12), ("p3_32", 4)])
def test_relax_candidates(name, r):
    gasa = _gasa()
    pr = problem(name)
    A = pr.A
    S = A.to_scipy()
    up = np.arange(A.n + 1) * A.b
    Dinv = O.invert_blocks(O.block_diagonal(S, up))
    W = Dinv.scaled(0.7)
    B0 = pr.B0[:, :r]
    Bw, sw = O.relax_candidates(S, W, B0, 0.03, 100)
    dB = to_dev(np.asfortranarray(B0).ravel(order="F"))
    got_sw = gasa.gasa_relax_candidates(A.n, A.b, to_dev(A.row_ptr), to_dev(A.col), to_dev(A.val.ravel()),
                                        to_dev(W.blocks.ravel()), dB, r, 0.03, 100)
    np.testing.assert_array_equal(got_sw, sw)
    Bg = to_host(dB).reshape(r, -1).T
    assert rel_err(Bg, Bw) <= 1e-11


@pytest.mark.parametrize("n_units,bs,size,r,s_next,seed", [
    (512, 3, 4, 12, 4, 41),      # P1 triangles, square blocks
    (256, 10, 4, 4, 4, 42),      # P3, r = 4 keeps everything
    (96, 10, 8, 80, 13, 43),     # P2 tets: 80 x 80 blocks, keep 13
    (101, 5, 4, 12, 4, 44),      # ragged last aggregate (5 rows)
    (40, 13, 8, 80, 17, 45),     # 104 x 80 blocks
])
def test_tentative(n_units, bs, size, r, s_next, seed):
    gasa = _gasa()
    B = np.asfortranarray(RO.random_normal(n_units * bs * r, seed).reshape(r, -1).T)
    agg = RO.chunk_aggregates(n_units, size)
    n_agg = int(agg.max()) + 1
    up = np.arange(n_units + 1) * bs
    rows = np.bincount(agg) * bs
    keep = [int(min(s_next, rj)) for rj in rows]
    Tw, _, sv = O.tentative(B, agg, up, n_agg, 3.0, keep=keep)
    T = to_dev(np.zeros(n_units * bs * s_next))
    sig = to_dev(np.zeros(n_agg * r))
    gasa.gasa_tentative(n_units, bs, n_agg, to_dev(agg), to_dev(B.ravel(order="F")), r, s_next, T, sig)
    Tg = to_host(T).reshape(n_units * bs, s_next)
    # dense oracle T, columns of aggregate J at offsets J*s_next (equal keep counts)
    Td = Tw.toarray()
    full = [J for J in range(n_agg) if keep[J] == s_next]
    for J in full:
        cols = slice(int(np.sum(keep[:J])), int(np.sum(keep[:J])) + s_next)
        rws = np.nonzero(agg == J)[0]
        rr = (rws[:, None] * bs + np.arange(bs)).ravel()
        sj = sv[J]
        # tolerance scales with eps / (relative singular-value gap) of the kept set
        gaps = np.abs(np.diff(sj[: min(len(sj), s_next + 1)])) / sj[0]
        tol = max(1e-11, 1e-13 / max(np.min(gaps), 1e-16))
        assert rel_err(Tg[rr], Td[rr, cols]) <= tol, J
    sg = to_host(sig).reshape(n_agg, r)
    for J in range(n_agg):
        k = min(r, len(sv[J]))
        assert rel_err(sg[J, :k], sv[J][:k]) <= 1e-12


@pytest.mark.parametrize("rank,s_next", [(2, 4), (1, 3), (0, 2)])
def test_tentative_rank_deficient_blocks(rank, s_next):
    """Candidate blocks of lower numerical rank than the kept count: the
    kept vectors with zero singular value are completed the same way on
    both sides (Gram-Schmidt of unit vectors), so T agrees column by column."""
    gasa = _gasa()
    n_units, bs, r, size = 64, 3, 12, 4
    n = n_units * bs
    if rank:
        B = RO.random_normal(n * rank, 71).reshape(n, rank) @ RO.random_normal(rank * r, 72).reshape(rank, r)
    else:
        B = np.zeros((n, r))
    B = np.asfortranarray(B)
    agg = RO.chunk_aggregates(n_units, size)
    n_agg = n_units // size
    up = np.arange(n_units + 1) * bs
    Tw, _, _ = O.tentative(B, agg, up, n_agg, 3.0, keep=[s_next] * n_agg)
    T = to_dev(np.zeros(n * s_next))
    gasa.gasa_tentative(n_units, bs, n_agg, to_dev(agg), to_dev(B.ravel(order="F")), r, s_next, T)
    Tg = to_host(T).reshape(n, s_next)
    Td = np.zeros((n, s_next))
    Tw = Tw.tocsr()
    for J in range(n_agg):
        rows = np.arange(J * size * bs, (J + 1) * size * bs)
        Td[rows] = Tw[rows][:, J * s_next:(J + 1) * s_next].toarray()
    assert np.max(np.abs(Tg - Td)) <= 1e-10
    for J in range(n_agg):
        rows = np.arange(J * size * bs, (J + 1) * size * bs)
        TJ = Tg[rows]
        assert np.max(np.abs(TJ.T @ TJ - np.eye(s_next))) <= 1e-13


@pytest.mark.parametrize("n", [1, 8, 192, 517])
def test_dense_inverse(n):
    gasa = _gasa()
    M = RO.random_blocks(1, n, 51)[0] + n * np.eye(n)
    Ainv = to_dev(np.zeros(n * n))
    sing = gasa.gasa_dense_inverse(n, to_dev(M.ravel()), Ainv)
    assert sing == 0
    X = to_host(Ainv).reshape(n, n)
    assert np.max(np.abs(X @ M - np.eye(n))) <= 1e-12


# FP32 blocks wider than 8 with >= 8 blocks per block row take the team-of-warps
# kernel (kernels_wide.cu): lane groups of br lanes (2 groups for 13 rows, 1 for
# 17..32, two rows per lane beyond 32), 1 to 8 warps per block row by the row
# length, rectangular restriction- and prolongation-shaped blocks
CASES_WIDE = [
    # (n_rows, n_cols, br, bc, per_row, seed)
    (100, 300, 5, 10, 24, 51),
    (64, 64, 36, 36, 16, 52),
    (50, 40, 13, 17, 30, 53),
    (33, 900, 4, 10, 70, 54),
    (40, 40, 16, 16, 12, 55),
    (20, 20, 32, 32, 11, 56),
    (301, 301, 12, 12, 19, 57),
    (80, 80, 22, 22, 100, 58),
    (131, 600, 13, 10, 9, 59),
    (60, 60, 40, 40, 10, 60),
    (2003, 2003, 9, 9, 10, 61),
]


@pytest.mark.parametrize("case", CASES_WIDE)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_bsr_mv_fp32_wide_blocks(case, mode):
    gasa = _gasa()
    n, m, br, bc, per, seed = case
    ptr, col, val = RO.random_bsr(n, m, br, bc, per, seed)
    assert ptr[-1] >= 8 * n
    x = RO.random_vector(m * bc, seed)
    b = RO.random_vector(n * br, seed, stream=120)
    y0 = RO.random_vector(n * br, seed, stream=121)
    Ax = bsr_scipy(ptr, col, val, m) @ x
    want = {0: Ax, 1: b - Ax, 2: y0 + Ax}[mode]
    y = to_dev(y0.astype(np.float32))
    f = np.float32
    gasa.gasa_bsr_mv_f32(mode, n, br, bc, to_dev(ptr), to_dev(col), to_dev(val.ravel().astype(f)),
                         to_dev(x.astype(f)), to_dev(b.astype(f)), y)
    assert rel_err(to_host(y), want) <= TOL32


@pytest.mark.parametrize("n,bs,seed,per_row", [(301, 12, 71, 19), (80, 22, 72, 100), (64, 36, 73, 16),
                                               (60, 40, 74, 10), (2003, 9, 75, 10), (129, 13, 76, 40)])
def test_jacobi_sweep_fp32_wide_blocks(n, bs, seed, per_row):
    gasa = _gasa()
    ptr, col, val, W, x, b = _jacobi_inputs(n, bs, seed, per_row)
    assert ptr[-1] >= 8 * n
    A = bsr_scipy(ptr, col, val)
    want = O.smooth_step(x, A, O.BlockDiag(np.arange(n + 1) * bs, W), b)
    out = to_dev(np.zeros(n * bs, np.float32))
    f = np.float32
    gasa.gasa_jacobi_sweep_f32(n, bs, to_dev(ptr), to_dev(col), to_dev(val.ravel().astype(f)),
                               to_dev(W.ravel().astype(f)), to_dev(x.astype(f)), to_dev(b.astype(f)), out)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(to_host(out) - want)) / scale <= 1e-4
