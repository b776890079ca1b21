"""Shared helpers of the test suite: cached workloads, cached oracle runs,
and device-buffer plumbing for the CUDA path (torch is used only to hold
device memory)."""
import functools

import numpy as np

from oracle import gasa_oracle as O
from synth import configs


@functools.lru_cache(maxsize=None)
def problem(name: str):
    if name == "c1":
        return configs.poisson2d_p1()
    if name == "p3_32":
        return configs.poisson2d_p3(n=32)
    if name == "p3_16":
        return configs.poisson2d_p3(n=16)
    if name == "tet_p2_4":
        # 384 tets: levels L0..L2 (a third coarsening would leave one aggregate)
        return configs.poisson3d(4, 2, r=80, n_levels=3, name="tet_p2_4")
    if name == "tet_p2_6":
        return configs.poisson3d(6, 2, r=80, n_levels=4, name="tet_p2_6")
    if name == "tiny":
        return configs.poisson2d(8, 1, r=12, n_levels=3, name="tiny")
    if name == "c2":
        return configs.poisson2d_p3()
    if name == "cd_q2_16":
        return configs.convdiff2d_q2(n=16, peclet=100.0)
    if name == "cd_q2_32_pe1e4":
        return configs.convdiff2d_q2(n=32, peclet=1e4)
    if name == "cd_q2_32_pe1":
        return configs.convdiff2d_q2(n=32, peclet=1.0)
    if name == "uneq6":
        # 72 triangles: level-2 aggregates hold 4, 4, 4, 4 and 2 units, so their
        # kept counts differ and level 2 is stored padded
        return configs.poisson2d(6, 1, r=12, n_levels=3, name="uneq6")
    if name == "p2_8":
        return configs.poisson2d(8, 2, r=24, n_levels=3, name="p2_8")
    if name.startswith("hex_M"):
        return configs.poisson3d_hex(int(name[5:]))
    if name.startswith("hexldg_M"):
        return configs.poisson3d_hex(int(name[8:]), flux="ldg")
    if name.startswith("cd3_"):
        # 3-D LDG + upwind on Kuhn tets, P1: cd3_<cells>_pe<Pe>
        _, n, pe = name.split("_")
        return configs.convdiff3d(int(n), 1, float(pe[2:]), name=name)
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def oracle_setup(name: str, cand_init: str = "R"):
    pr = problem(name)
    A = pr.A
    return O.setup(A.row_ptr, A.col, A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=pr.dim,
                   cand_init=cand_init)


def torch_dev():
    import torch
    assert torch.cuda.is_available(), "CUDA device required"
    return torch.device("cuda:0")


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch_dev())


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_setup(name: str, keep: bool = True, **opt_kw):
    from paper_2504_13373_gb300 import gasa
    pr = problem(name)
    A = pr.A
    ctx = gasa.gasa_create(0)
    kw = dict(dim=pr.dim, n_cand=pr.r, keep_setup_data=1 if keep else 0,
              solver=gasa.GASA_SOLVER_CG if pr.solver == "cg" else gasa.GASA_SOLVER_GMRES)
    kw.update(opt_kw)
    opt = gasa.gasa_default_options(**kw)
    info = gasa.gasa_setup(ctx, A.row_ptr, A.col, A.val.ravel(), A.b, pr.agg_of, opt,
                           adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx, centroids=pr.centroids,
                           init_candidates=pr.B0)
    return ctx, info


def bsr_scipy(ptr, col, val, n_cols_blocks=None):
    import scipy.sparse as sp
    n = ptr.size - 1
    br, bc = val.shape[1], val.shape[2]
    nc = n_cols_blocks if n_cols_blocks is not None else n
    return sp.bsr_matrix((val, col, ptr), shape=(n * br, nc * bc)).tocsr()


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.max(np.abs(a - b)) if a.size else 0.0
    s = np.max(np.abs(b)) if b.size else 0.0
    return d / s if s > 0 else d
