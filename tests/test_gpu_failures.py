"""Failure paths of the C ABI, each fault made on the host: malformed inputs
that gasa_setup must reject before any device work, a zeroed diagonal block
(the block-Jacobi smoother of Eq. smoother_choice needs D_k^{-1}), a
non-finite right-hand side, an iteration limit, and a served request with a
non-finite right-hand side beside healthy ones.  Every case must return its
status (and never hang); nothing here faults or traps the GPU."""
import numpy as np
import pytest

from synth import configs, serving
from tests.helpers import problem

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _gasa():
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    return gasa


def _setup_status(gasa, pr, row_ptr=None, col=None, val=None, adj_ptr=None, adj_idx=None,
                  **opt_kw):
    A = pr.A
    row_ptr = A.row_ptr if row_ptr is None else row_ptr
    col = A.col if col is None else col
    val = A.val if val is None else val
    adj_ptr = pr.adj_ptr if adj_ptr is None else adj_ptr
    adj_idx = pr.adj_idx if adj_idx is None else adj_idx
    ctx = gasa.gasa_create(0)
    try:
        opt = gasa.gasa_default_options(dim=pr.dim, n_cand=pr.r, **opt_kw)
        try:
            gasa.gasa_setup(ctx, row_ptr, col, np.ascontiguousarray(val).ravel(), A.b, pr.agg_of,
                            opt, adj_ptr=adj_ptr, adj_idx=adj_idx, centroids=pr.centroids,
                            init_candidates=pr.B0)
            return gasa.GASA_OK, ""
        except gasa.GasaError as e:
            return e.status, str(e)
    finally:
        gasa.gasa_destroy(ctx)


def _row_with_blocks(A, at_least=3):
    counts = np.diff(A.row_ptr)
    return int(np.nonzero(counts >= at_least)[0][0])


def test_setup_rejects_unsorted_columns():
    gasa = _gasa()
    pr = problem("tiny")
    A = pr.A
    i = _row_with_blocks(A)
    a = A.row_ptr[i]
    col, val = A.col.copy(), A.val.copy()
    col[[a, a + 1]] = col[[a + 1, a]]
    val[[a, a + 1]] = val[[a + 1, a]]
    st, msg = _setup_status(gasa, pr, col=col, val=val)
    assert st == gasa.GASA_ERR_INVALID_ARG and "increasing" in msg, msg


def test_setup_rejects_missing_diagonal_block():
    gasa = _gasa()
    pr = problem("tiny")
    A = pr.A
    i = _row_with_blocks(A)
    a, b = A.row_ptr[i], A.row_ptr[i + 1]
    d = a + int(np.nonzero(A.col[a:b] == i)[0][0])
    keep = np.ones(A.col.size, bool)
    keep[d] = False
    row_ptr = A.row_ptr.copy()
    row_ptr[i + 1:] -= 1
    st, msg = _setup_status(gasa, pr, row_ptr=row_ptr, col=A.col[keep], val=A.val[keep])
    assert st == gasa.GASA_ERR_INVALID_ARG and "diagonal" in msg, msg


def test_setup_rejects_out_of_range_column():
    gasa = _gasa()
    pr = problem("tiny")
    A = pr.A
    last = A.row_ptr[-1] - 1              # last block of the last row: raise its column past n
    col = A.col.copy()
    col[last] = A.n
    st, msg = _setup_status(gasa, pr, col=col)
    assert st == gasa.GASA_ERR_INVALID_ARG and "range" in msg, msg


def test_setup_rejects_asymmetric_adjacency():
    gasa = _gasa()
    pr = problem("tiny")
    ap, ai = pr.adj_ptr.astype(np.int64), pr.adj_idx
    i = 0
    drop = ap[i]                          # the edge i -> ai[ap[i]], keeping its reverse
    keep = np.ones(ai.size, bool)
    keep[drop] = False
    ap2 = ap.copy()
    ap2[i + 1:] -= 1
    st, msg = _setup_status(gasa, pr, adj_ptr=ap2.astype(np.int32), adj_idx=ai[keep])
    assert st == gasa.GASA_ERR_INVALID_ARG and "symmetric" in msg, msg


def test_setup_reports_a_zeroed_diagonal_block():
    gasa = _gasa()
    pr = problem("tiny")
    A = pr.A
    i = 5
    a, b = A.row_ptr[i], A.row_ptr[i + 1]
    d = a + int(np.nonzero(A.col[a:b] == i)[0][0])
    val = A.val.copy()
    val[d] = 0.0
    st, msg = _setup_status(gasa, pr, val=val)
    assert st == gasa.GASA_ERR_SINGULAR_BLOCK, msg


def _ctx(gasa, name, **kw):
    from tests.helpers import gpu_setup
    return gpu_setup(name, keep=False, **kw)[0]


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_nonfinite_rhs_is_a_breakdown(precision):
    """A NaN entry in b: CG stops with GASA_ERR_BREAKDOWN (each precision);
    the context stays usable for the next, healthy solve."""
    gasa = _gasa()
    pr = problem("c1")
    ctx = _ctx(gasa, "c1")
    try:
        b = pr.rhs.copy()
        b[17] = np.nan
        x = np.zeros_like(b)
        with pytest.raises(gasa.GasaError) as ei:
            gasa.gasa_solve(ctx, b, x, TOL, precision)
        assert ei.value.status == gasa.GASA_ERR_BREAKDOWN
        info = gasa.gasa_solve(ctx, pr.rhs, x, TOL, precision)
        assert info.converged and info.rel_residual <= TOL
    finally:
        gasa.gasa_destroy(ctx)


def test_nonfinite_rhs_gmres_is_a_breakdown():
    gasa = _gasa()
    pr = problem("cd_q2_16")
    ctx = _ctx(gasa, "cd_q2_16", solver=gasa.GASA_SOLVER_GMRES)
    try:
        b = pr.rhs.copy()
        b[3] = np.inf
        x = np.zeros_like(b)
        with pytest.raises(gasa.GasaError) as ei:
            gasa.gasa_solve(ctx, b, x, TOL)
        assert ei.value.status == gasa.GASA_ERR_BREAKDOWN
    finally:
        gasa.gasa_destroy(ctx)


def test_iteration_limit_reports_not_converged_and_writes_x():
    """max_iter = 3: GASA_ERR_NOT_CONVERGED, x holds the third iterate and
    the reported residual is its true residual."""
    gasa = _gasa()
    pr = problem("c1")
    ctx = _ctx(gasa, "c1", max_iter=3)
    try:
        x = np.full_like(pr.rhs, np.nan)
        info = gasa.gasa_solve(ctx, pr.rhs, x, TOL, allow_not_converged=True)
        assert info.iterations == 3 and not info.converged
        assert np.all(np.isfinite(x))
        rel = np.linalg.norm(pr.rhs - pr.A.to_scipy() @ x) / np.linalg.norm(pr.rhs)
        assert TOL < rel < 1.0
        assert abs(rel - info.rel_residual) <= 1e-10 * rel
        with pytest.raises(gasa.GasaError) as ei:
            gasa.gasa_solve(ctx, pr.rhs, x, TOL)
        assert ei.value.status == gasa.GASA_ERR_NOT_CONVERGED
    finally:
        gasa.gasa_destroy(ctx)


def test_served_nonfinite_request_leaves_batch_mates_unchanged():
    """One served request with a NaN right-hand side among healthy ones on
    the same engine: it ends with GASA_ERR_BREAKDOWN, and every healthy
    request gives the same bits and iterations as when served alone."""
    gasa = _gasa()
    pr = problem("c1")
    ctx = _ctx(gasa, "c1")
    n = pr.n_dofs
    rhs = [serving.request_rhs(configs.SEED, i, n) for i in range(3)]
    bad = rhs[1].copy()
    bad[100] = np.nan

    def serve(batch, max_batch):
        srv = gasa.gasa_server_create(0, 4 << 30, max_batch)
        try:
            mid = gasa.gasa_server_add_mesh(srv, ctx)
            ts = [gasa.gasa_server_submit(srv, mid, b, TOL, gasa.GASA_PREC_MIXED32) for b in batch]
            gasa.gasa_server_drain(srv, 300.0)
            out = []
            for t in ts:
                x = np.zeros(n)
                st, info = gasa.gasa_server_poll(srv, t, x)
                out.append((st, info.iterations, x))
            return out
        finally:
            gasa.gasa_server_destroy(srv)

    try:
        alone = [serve([b], 1)[0] for b in (rhs[0], rhs[2])]
        mixed = serve([rhs[0], bad, rhs[2]], 4)
        assert mixed[1][0] == gasa.GASA_ERR_BREAKDOWN
        for want, got in zip(alone, (mixed[0], mixed[2])):
            assert want[0] == got[0] == gasa.GASA_OK
            assert want[1] == got[1]
            assert np.array_equal(want[2], got[2])
    finally:
        gasa.gasa_destroy(ctx)
