"""Request server (continuous batching of solves on resident hierarchies).

* a served solve matches the CPU oracle like a single solve: iteration count
  within 1, FP64 solution within 1e-10 relative, true residual <= 1e-10;
* a request gives the same bits alone and in a mix of meshes, precisions,
  slots and batch widths, with requests joining while others run;
* the HBM budget admits hierarchies and engines, and engines without work
  are released so that waiting requests can run.
"""
import time

import numpy as np
import pytest

from oracle import gasa_oracle as O
from synth import configs, serving
from tests.helpers import gpu_setup, oracle_setup, problem

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _gasa():
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    return gasa


def _finish(gasa, srv, ticket, n):
    x = np.zeros(n)
    st, info = gasa.gasa_server_poll(srv, ticket, x)
    assert st == gasa.GASA_OK, (st, gasa.gasa_status_string(st), gasa.gasa_server_last_error(srv))
    assert info.converged == 1 and info.rel_residual <= TOL
    return x, info


@pytest.mark.parametrize("name", ["c1", "cd_q2_16"])
def test_served_solve_matches_oracle(name):
    gasa = _gasa()
    pr = problem(name)
    H = oracle_setup(name)
    ref = O.solve(H, pr.rhs, TOL, pr.solver, restart=30, max_iter=5000)
    ref32 = O.solve(H, pr.rhs, TOL, pr.solver, precision="mixed32", restart=30, max_iter=5000)
    ref16 = O.solve(H, pr.rhs, TOL, pr.solver, precision="mixed16", restart=30, max_iter=5000)
    ctx, _ = gpu_setup(name, keep=False)
    srv = gasa.gasa_server_create(0, 8 << 30, 8)
    try:
        mid = gasa.gasa_server_add_mesh(srv, ctx)
        t64 = gasa.gasa_server_submit(srv, mid, pr.rhs, TOL, gasa.GASA_PREC_FP64)
        t32 = gasa.gasa_server_submit(srv, mid, pr.rhs, TOL, gasa.GASA_PREC_MIXED32)
        t16 = gasa.gasa_server_submit(srv, mid, pr.rhs, TOL, gasa.GASA_PREC_MIXED16)
        gasa.gasa_server_drain(srv, 300.0)
        x, info = _finish(gasa, srv, t64, pr.n_dofs)
        assert abs(info.iterations - ref.iterations) <= 1, (info.iterations, ref.iterations)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= TOL
        xm, info32 = _finish(gasa, srv, t32, pr.n_dofs)
        assert abs(info32.iterations - ref32.iterations) <= 1, (info32.iterations, ref32.iterations)
        A = pr.A.to_scipy()
        assert np.linalg.norm(pr.rhs - A @ xm) / np.linalg.norm(pr.rhs) <= TOL
        # FP16-block level 0: the oracle's FP16 emulation of the same storage
        xh, info16 = _finish(gasa, srv, t16, pr.n_dofs)
        assert abs(info16.iterations - ref16.iterations) <= 1, (info16.iterations, ref16.iterations)
        assert np.linalg.norm(pr.rhs - A @ xh) / np.linalg.norm(pr.rhs) <= TOL
    finally:
        gasa.gasa_server_destroy(srv)
        gasa.gasa_destroy(ctx)


MIX = ["c1", "tiny", "cd_q2_16", "tet_p2_4"]


def _contexts(gasa):
    return {name: gpu_setup(name, keep=False)[0] for name in MIX}


def _alone(gasa, ctxs, max_batch, jobs):
    """Each job (mesh name, precision, rhs index) solved with nothing else in flight."""
    srv = gasa.gasa_server_create(0, 16 << 30, max_batch)
    out = {}
    try:
        ids = {name: gasa.gasa_server_add_mesh(srv, ctxs[name]) for name in MIX}
        for name, prec, i in jobs:
            n = problem(name).n_dofs
            t = gasa.gasa_server_submit(srv, ids[name], serving.request_rhs(configs.SEED, i, n), TOL, prec)
            gasa.gasa_server_drain(srv, 300.0)
            out[(name, prec, i)] = _finish(gasa, srv, t, n)
        stats = gasa.gasa_server_stats_read(srv)
    finally:
        gasa.gasa_server_destroy(srv)
    return out, stats


def _mix(gasa, ctxs, max_batch, jobs, budget=16 << 30, pause=0.002):
    srv = gasa.gasa_server_create(0, budget, max_batch)
    out = {}
    try:
        ids = {name: gasa.gasa_server_add_mesh(srv, ctxs[name]) for name in MIX}
        tickets = {}
        for k, (name, prec, i) in enumerate(jobs):
            n = problem(name).n_dofs
            tickets[(name, prec, i)] = gasa.gasa_server_submit(
                srv, ids[name], serving.request_rhs(configs.SEED, i, n), TOL, prec)
            if k % 5 == 4:
                time.sleep(pause)       # later requests join running batches
        gasa.gasa_server_drain(srv, 600.0)
        for key, t in tickets.items():
            out[key] = _finish(gasa, srv, t, problem(key[0]).n_dofs)
        stats = gasa.gasa_server_stats_read(srv)
    finally:
        gasa.gasa_server_destroy(srv)
    return out, stats


def _jobs(gasa, idx):
    jobs = [(name, prec, i) for i in idx for name in MIX
            for prec in (gasa.GASA_PREC_FP64, gasa.GASA_PREC_MIXED32, gasa.GASA_PREC_MIXED16)]
    order = np.argsort(serving.request_mesh(configs.SEED, len(jobs), 997), kind="stable")
    return [jobs[k] for k in order]


def test_same_bits_alone_and_in_the_mix():
    gasa = _gasa()
    ctxs = _contexts(gasa)
    try:
        base = _jobs(gasa, [0])
        alone, _ = _alone(gasa, ctxs, 8, base)
        mixed, stats = _mix(gasa, ctxs, 4, _jobs(gasa, [0, 1, 2, 3]))
        assert stats["completed"] == stats["submitted"] == 4 * len(base)
        assert stats["peak_running"] >= 2          # solves overlapped on the device
        narrow, _ = _mix(gasa, ctxs, 1, _jobs(gasa, [0, 1]))
        for key, (x, info) in alone.items():
            for other in (mixed, narrow):
                y, inf2 = other[key]
                assert inf2.iterations == info.iterations, key
                assert np.array_equal(x, y), key
        # different right-hand sides give different answers (the mix is real)
        k0 = ("c1", gasa.GASA_PREC_FP64, 0)
        assert not np.array_equal(mixed[k0][0], mixed[("c1", gasa.GASA_PREC_FP64, 1)][0])
    finally:
        for c in ctxs.values():
            gasa.gasa_destroy(c)


def test_budget_releases_idle_engines():
    gasa = _gasa()
    ctxs = _contexts(gasa)
    try:
        # engine sizes at one slot, from a server with room for everything
        probe = gasa.gasa_server_create(0, 16 << 30, 1)
        try:
            for name in MIX:
                gasa.gasa_server_add_mesh(probe, ctxs[name])
            used0 = gasa.gasa_server_stats_read(probe)["used_bytes"]
            sizes = []
            jobs = _jobs(gasa, [0])
            for k, (name, prec, i) in enumerate(jobs):
                before = gasa.gasa_server_stats_read(probe)["used_bytes"]
                n = problem(name).n_dofs
                t = gasa.gasa_server_submit(probe, MIX.index(name),
                                            serving.request_rhs(configs.SEED, i, n), TOL, prec)
                gasa.gasa_server_drain(probe, 300.0)
                _finish(gasa, probe, t, n)
                sizes.append(gasa.gasa_server_stats_read(probe)["used_bytes"] - before)
        finally:
            gasa.gasa_server_destroy(probe)
        alone, _ = _alone(gasa, ctxs, 8, jobs)
        budget = used0 + max(sizes)        # one single-slot engine at a time
        out, stats = _mix(gasa, ctxs, 8, _jobs(gasa, [0, 1]), budget=budget)
        assert stats["engines_released"] >= 1
        assert stats["peak_bytes"] <= budget
        for key, (x, info) in alone.items():
            assert np.array_equal(out[key][0], x), key
        # a hierarchy that does not fit is refused
        small = gasa.gasa_server_create(0, 1024, 8)
        try:
            with pytest.raises(gasa.GasaError) as ei:
                gasa.gasa_server_add_mesh(small, ctxs["c1"])
            assert ei.value.status == gasa.GASA_ERR_BUDGET
        finally:
            gasa.gasa_server_destroy(small)
    finally:
        for c in ctxs.values():
            gasa.gasa_destroy(c)


def test_server_requests_validated():
    gasa = _gasa()
    ctx, _ = gpu_setup("tiny", keep=False)
    srv = gasa.gasa_server_create(0, 1 << 30, 2)
    try:
        mid = gasa.gasa_server_add_mesh(srv, ctx)
        n = problem("tiny").n_dofs
        with pytest.raises(gasa.GasaError) as ei:
            gasa.gasa_server_submit(srv, mid, np.ones(n), TOL, 7)     # no such precision
        assert ei.value.status == gasa.GASA_ERR_INVALID_ARG
        with pytest.raises(gasa.GasaError):
            gasa.gasa_server_submit(srv, mid + 1, np.ones(n), TOL, gasa.GASA_PREC_FP64)
        with pytest.raises(gasa.GasaError):
            gasa.gasa_server_poll(srv, 12345)
        t = gasa.gasa_server_submit(srv, mid, np.zeros(n), TOL, gasa.GASA_PREC_FP64)
        x = np.ones(n)
        st, info = gasa.gasa_server_poll(srv, t, x)
        assert st == gasa.GASA_OK and not x.any()
        t = gasa.gasa_server_submit(srv, mid, problem("tiny").rhs, TOL, gasa.GASA_PREC_FP64)
        st, _ = gasa.gasa_server_poll(srv, t)
        assert st in (gasa.GASA_PENDING, gasa.GASA_OK)
        gasa.gasa_server_drain(srv, 60.0)
        st, info = gasa.gasa_server_poll(srv, t)
        assert st == gasa.GASA_OK and info.rel_residual <= TOL
    finally:
        gasa.gasa_server_destroy(srv)
        gasa.gasa_destroy(ctx)
