"""Python binding of the C ABI in include/gasa.h (argument marshalling only).

Every function keeps the C name.  Host arrays are numpy arrays; device
arrays are anything with `data_ptr()` (torch CUDA tensors) or raw integer
addresses.  Statuses other than GASA_OK raise `GasaError` unless the call is
documented to return it.  There is no fallback: if libgasa.so is missing the
import of this module's functions fails loudly.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgasa.so")

GASA_OK = 0
GASA_ERR_INVALID_ARG = 1
GASA_ERR_OOM = 2
GASA_ERR_CUDA = 3
GASA_ERR_SINGULAR_BLOCK = 4
GASA_ERR_NOT_SPD = 5
GASA_ERR_NOT_CONVERGED = 6
GASA_ERR_BREAKDOWN = 7
GASA_ERR_TIMEOUT = 8
GASA_ERR_BUDGET = 9
GASA_PENDING = 10
GASA_ERR_UNSUPPORTED = 11
GASA_ERR_STATE = 12

GASA_SOLVER_CG, GASA_SOLVER_GMRES, GASA_SOLVER_STATIONARY = 0, 1, 2
GASA_PREC_FP64, GASA_PREC_MIXED32, GASA_PREC_MIXED16 = 0, 1, 2
GASA_CAND_R, GASA_CAND_TT = 0, 1
GASA_MV_ASSIGN, GASA_MV_RESIDUAL, GASA_MV_ADD = 0, 1, 2
GASA_MAX_LEVELS = 24

(GASA_LV_A_ROWPTR, GASA_LV_A_COL, GASA_LV_A_VAL, GASA_LV_P_ROWPTR, GASA_LV_P_COL, GASA_LV_P_VAL,
 GASA_LV_R_ROWPTR, GASA_LV_R_COL, GASA_LV_R_VAL, GASA_LV_T_VAL, GASA_LV_W, GASA_LV_CAND,
 GASA_LV_SWEEPS, GASA_LV_COARSE_INV, GASA_LV_CAND_IN, GASA_LV_SIZES, GASA_LV_RA_ROWPTR,
 GASA_LV_RA_COL, GASA_LV_RA_VAL, GASA_LV_DENSE_TAIL, GASA_LV_WA) = range(21)

# every symbol include/gasa.h declares
EXPORTS = [
    "gasa_default_options", "gasa_create", "gasa_setup", "gasa_solve", "gasa_vcycle",
    "gasa_level_shape", "gasa_tail_info", "gasa_cycle_info", "gasa_get_level", "gasa_profile_enable", "gasa_profile_read",
    "gasa_destroy", "gasa_status_string", "gasa_last_error", "gasa_bsr_mv", "gasa_bsr_mv_f32", "gasa_bsr_mv_ds",
    "gasa_jacobi_sweep", "gasa_jacobi_sweep_f32", "gasa_block_inverse", "gasa_power_estimate",
    "gasa_relax_candidates", "gasa_tentative", "gasa_dense_inverse", "gasa_kernel_launches",
    "gasa_power_estimate_noalloc",
    "gasa_server_create", "gasa_server_add_mesh", "gasa_server_submit", "gasa_server_poll",
    "gasa_server_drain", "gasa_server_stats_read", "gasa_server_destroy", "gasa_server_last_error",
]
GASA_NOALLOC_MAX_DOFS = 262144

c_i32, c_i64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class gasa_bsr(ctypes.Structure):
    _fields_ = [("n_blocks", c_i32), ("block", c_i32), ("nnzb", c_i32),
                ("row_ptr", c_vp), ("col", c_vp), ("val", c_vp), ("on_device", c_i32)]


class gasa_hierarchy(ctypes.Structure):
    _fields_ = [("n_levels", c_i32), ("agg_of", ctypes.POINTER(c_vp))]


class gasa_options(ctypes.Structure):
    _fields_ = [("dim", c_i32), ("solver", c_i32), ("restart", c_i32), ("precision", c_i32),
                ("t_pre", c_i32), ("t_post", c_i32), ("q_power", c_i32), ("n_cand", c_i32),
                ("max_relax", c_i32), ("max_iter", c_i32), ("cand_init", c_i32),
                ("keep_setup_data", c_i32), ("gamma", c_dbl), ("omega_factor", c_dbl),
                ("n_cut", c_dbl), ("seed", ctypes.c_uint64), ("init_candidates", c_vp),
                ("bulk_staging", c_i32), ("matrix_free_levels", c_i32), ("hstar", c_i32),
                ("delta", c_dbl), ("tail_kib", c_i32), ("grid_tail", c_i32),
                ("wait_budget_s", c_dbl), ("fused_restriction", c_i32),
                ("dense_tail_dofs", c_i32), ("folded_smoother", c_i32)]


class gasa_setup_info(ctypes.Structure):
    _fields_ = [("n_levels", c_i32), ("n_cand", c_i32),
                ("units", c_i64 * GASA_MAX_LEVELS), ("block", c_i32 * GASA_MAX_LEVELS),
                ("dofs", c_i64 * GASA_MAX_LEVELS), ("nnzb", c_i64 * GASA_MAX_LEVELS),
                ("nnz", c_i64 * GASA_MAX_LEVELS), ("omega", c_dbl * GASA_MAX_LEVELS),
                ("rho", c_dbl * GASA_MAX_LEVELS), ("relax_sweeps_max", c_i32 * GASA_MAX_LEVELS),
                ("seconds", c_dbl), ("device_bytes", c_i64)]


class gasa_solve_info(ctypes.Structure):
    _fields_ = [("iterations", c_i32), ("converged", c_i32), ("rel_residual", c_dbl),
                ("seconds", c_dbl)]


class gasa_server_stats(ctypes.Structure):
    _fields_ = [(k, c_i64) for k in (
        "submitted", "completed", "queued", "running", "engines", "engines_created",
        "engines_released", "budget_bytes", "used_bytes", "peak_bytes", "peak_running",
        "graph_launches")]


class GasaError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"gasa status {status}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libgasa.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.gasa_status_string.restype = ctypes.c_char_p
    L.gasa_last_error.restype = ctypes.c_char_p
    L.gasa_server_last_error.restype = ctypes.c_char_p
    L.gasa_default_options.restype = None
    L.gasa_kernel_launches.restype = ctypes.c_int64
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("gasa_status_string", "gasa_last_error", "gasa_default_options",
                        "gasa_kernel_launches", "gasa_server_last_error"):
            f.restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    """Address of a numpy array, a tensor with data_ptr(), an int or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(f"cannot take the address of {type(a)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st, ctx=None, allow=()):
    if st == GASA_OK or st in allow:
        return st
    L = load()
    msg = L.gasa_status_string(st).decode()
    if ctx is not None:
        msg += ": " + L.gasa_last_error(ctx).decode()
    raise GasaError(st, msg)


def gasa_status_string(st):
    return load().gasa_status_string(st).decode()


def gasa_last_error(ctx):
    return load().gasa_last_error(ctx).decode()


def gasa_default_options(**kw):
    opt = gasa_options()
    load().gasa_default_options(ctypes.byref(opt))
    for k, v in kw.items():
        if not hasattr(opt, k):
            raise AttributeError(k)
        setattr(opt, k, v)
    return opt


def gasa_create(device=0, stream=None):
    ctx = c_vp()
    _check(load().gasa_create(ctypes.byref(ctx), c_i32(device), c_vp(_stream(stream))))
    return ctx


def gasa_setup(ctx, row_ptr, col, val, block, agg_of, options, adj_ptr=None, adj_idx=None,
               centroids=None, on_device=False, init_candidates=None):
    """row_ptr/col int32, val float64 (nnzb*block*block); agg_of: list of int32
    host arrays; init_candidates: host float64 n x r, column-major."""
    keep = []
    n = (row_ptr.shape[0] if hasattr(row_ptr, "shape") else len(row_ptr)) - 1
    nnzb = col.shape[0] if hasattr(col, "shape") else len(col)
    if not on_device:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        keep += [row_ptr, col, val]
    A = gasa_bsr(n, block, nnzb, _ptr(row_ptr), _ptr(col), _ptr(val), 1 if on_device else 0)
    aggs = [np.ascontiguousarray(a, dtype=np.int32) for a in agg_of]
    keep += aggs
    arr = (c_vp * len(aggs))(*[a.ctypes.data for a in aggs])
    H = gasa_hierarchy(len(aggs) + 1, ctypes.cast(arr, ctypes.POINTER(c_vp)))
    if adj_ptr is not None:
        adj_ptr = np.ascontiguousarray(adj_ptr, dtype=np.int32)
        adj_idx = np.ascontiguousarray(adj_idx, dtype=np.int32)
        keep += [adj_ptr, adj_idx]
    if centroids is not None:
        centroids = np.ascontiguousarray(centroids, dtype=np.float64)
        keep.append(centroids)
    if init_candidates is not None:
        init_candidates = np.asfortranarray(init_candidates, dtype=np.float64)
        keep.append(init_candidates)
        options.init_candidates = init_candidates.ctypes.data
    info = gasa_setup_info()
    st = load().gasa_setup(ctx, ctypes.byref(A), c_vp(_ptr(adj_ptr)), c_vp(_ptr(adj_idx)),
                           c_vp(_ptr(centroids)), ctypes.byref(H), ctypes.byref(options),
                           ctypes.byref(info))
    options.init_candidates = None
    _check(st, ctx)
    return info


def gasa_solve(ctx, b, x, tol, precision=GASA_PREC_FP64, on_device=False,
               allow_not_converged=False):
    info = gasa_solve_info()
    st = load().gasa_solve(ctx, c_vp(_ptr(b)), c_vp(_ptr(x)), c_dbl(tol), c_i32(precision),
                           c_i32(1 if on_device else 0), ctypes.byref(info))
    _check(st, ctx, allow=(GASA_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return info


def gasa_vcycle(ctx, r, z, precision=GASA_PREC_FP64):
    _check(load().gasa_vcycle(ctx, c_vp(_ptr(r)), c_vp(_ptr(z)), c_i32(precision)), ctx)


def gasa_level_shape(ctx, level):
    sh = (c_i64 * 8)()
    _check(load().gasa_level_shape(ctx, c_i32(level), sh), ctx)
    keys = ["units", "s", "nnzb", "P_nnzb", "R_nnzb", "s_next", "r", "dofs"]
    return dict(zip(keys, [int(v) for v in sh]))


def gasa_tail_info(ctx, precision):
    out = (c_i32 * 3)()
    _check(load().gasa_tail_info(ctx, c_i32(precision), out), ctx)
    return {"first_level": int(out[0]), "cluster": int(out[1]), "coarse_inside": int(out[2])}


def gasa_cycle_info(ctx):
    out = (c_i32 * 3)()
    _check(load().gasa_cycle_info(ctx, out), ctx)
    return {"dense_first_level": int(out[0]), "dense_n": int(out[1]), "folded": int(out[2])}


def gasa_get_level(ctx, level, what, out: np.ndarray):
    _check(load().gasa_get_level(ctx, c_i32(level), c_i32(what), c_vp(out.ctypes.data),
                                 c_i64(out.nbytes)), ctx)
    return out


def gasa_profile_enable(ctx, on=True):
    _check(load().gasa_profile_enable(ctx, c_i32(1 if on else 0)), ctx)


def gasa_profile_read(ctx, kernel_class):
    ms, n, by = c_dbl(), c_i64(), c_dbl()
    _check(load().gasa_profile_read(ctx, c_i32(kernel_class), ctypes.byref(ms), ctypes.byref(n),
                                    ctypes.byref(by)), ctx)
    return ms.value, n.value, by.value


def gasa_destroy(ctx):
    _check(load().gasa_destroy(ctx))


def gasa_kernel_launches():
    return int(load().gasa_kernel_launches())


# request server -----------------------------------------------------------------

def _check_srv(st, srv, allow=()):
    if st == GASA_OK or st in allow:
        return st
    L = load()
    raise GasaError(st, L.gasa_status_string(st).decode() + ": " +
                    L.gasa_server_last_error(srv).decode())


def gasa_server_create(device=0, budget_bytes=40 << 30, max_batch=8):
    srv = c_vp()
    _check(load().gasa_server_create(ctypes.byref(srv), c_i32(device), c_i64(budget_bytes),
                                     c_i32(max_batch)))
    return srv


def gasa_server_add_mesh(srv, ctx):
    mid = c_i32()
    _check_srv(load().gasa_server_add_mesh(srv, ctx, ctypes.byref(mid)), srv)
    return mid.value


def gasa_server_submit(srv, mesh_id, b, tol, precision=GASA_PREC_FP64):
    """b: host float64 array (copied before return); returns the ticket."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    t = ctypes.c_uint64()
    _check_srv(load().gasa_server_submit(srv, c_i32(mesh_id), c_vp(b.ctypes.data), c_dbl(tol),
                                         c_i32(precision), ctypes.byref(t)), srv)
    return t.value


def gasa_server_poll(srv, ticket, x_out=None):
    """(status, info); status GASA_PENDING while the solve is not finished.
    x_out: host float64 array of the mesh's dofs, written when finished."""
    info = gasa_solve_info()
    st = load().gasa_server_poll(srv, ctypes.c_uint64(ticket), c_vp(_ptr(x_out)), ctypes.byref(info))
    if st == GASA_ERR_INVALID_ARG:
        _check_srv(st, srv)
    return st, info


def gasa_server_drain(srv, timeout_s=600.0):
    _check_srv(load().gasa_server_drain(srv, c_dbl(timeout_s)), srv)


def gasa_server_stats_read(srv):
    out = gasa_server_stats()
    _check(load().gasa_server_stats_read(srv, ctypes.byref(out)))
    return {k: int(getattr(out, k)) for k, _ in gasa_server_stats._fields_}


def gasa_server_destroy(srv):
    _check(load().gasa_server_destroy(srv))


def gasa_server_last_error(srv):
    return load().gasa_server_last_error(srv).decode()


# single operations -------------------------------------------------------------

def gasa_bsr_mv(mode, n_brows, br, bc, row_ptr, col, val, x, b, y, stream=None):
    _check(load().gasa_bsr_mv(c_i32(mode), c_i32(n_brows), c_i32(br), c_i32(bc),
                              c_vp(_ptr(row_ptr)), c_vp(_ptr(col)), c_vp(_ptr(val)),
                              c_vp(_ptr(x)), c_vp(_ptr(b)), c_vp(_ptr(y)), c_vp(_stream(stream))))


def gasa_bsr_mv_f32(mode, n_brows, br, bc, row_ptr, col, val, x, b, y, stream=None):
    _check(load().gasa_bsr_mv_f32(c_i32(mode), c_i32(n_brows), c_i32(br), c_i32(bc),
                                  c_vp(_ptr(row_ptr)), c_vp(_ptr(col)), c_vp(_ptr(val)),
                                  c_vp(_ptr(x)), c_vp(_ptr(b)), c_vp(_ptr(y)),
                                  c_vp(_stream(stream))))


def gasa_bsr_mv_ds(n_brows, br, bc, row_ptr, col, a_hi, a_lo, x_hi, x_lo, y, stream=None):
    _check(load().gasa_bsr_mv_ds(c_i32(n_brows), c_i32(br), c_i32(bc), c_vp(_ptr(row_ptr)),
                                 c_vp(_ptr(col)), c_vp(_ptr(a_hi)), c_vp(_ptr(a_lo)),
                                 c_vp(_ptr(x_hi)), c_vp(_ptr(x_lo)), c_vp(_ptr(y)),
                                 c_vp(_stream(stream))))


def gasa_jacobi_sweep(n_units, bs, row_ptr, col, val, W, x, b, x_out, first=False, stream=None):
    _check(load().gasa_jacobi_sweep(c_i32(n_units), c_i32(bs), c_vp(_ptr(row_ptr)),
                                    c_vp(_ptr(col)), c_vp(_ptr(val)), c_vp(_ptr(W)),
                                    c_vp(_ptr(x)), c_vp(_ptr(b)), c_vp(_ptr(x_out)),
                                    c_i32(1 if first else 0), c_vp(_stream(stream))))


def gasa_jacobi_sweep_f32(n_units, bs, row_ptr, col, val, W, x, b, x_out, first=False,
                          stream=None):
    _check(load().gasa_jacobi_sweep_f32(c_i32(n_units), c_i32(bs), c_vp(_ptr(row_ptr)),
                                        c_vp(_ptr(col)), c_vp(_ptr(val)), c_vp(_ptr(W)),
                                        c_vp(_ptr(x)), c_vp(_ptr(b)), c_vp(_ptr(x_out)),
                                        c_i32(1 if first else 0), c_vp(_stream(stream))))


def gasa_block_inverse(n_units, bs, row_ptr, col, val, scale, W_out, stream=None):
    ns = c_i32()
    _check(load().gasa_block_inverse(c_i32(n_units), c_i32(bs), c_vp(_ptr(row_ptr)),
                                     c_vp(_ptr(col)), c_vp(_ptr(val)), c_dbl(scale),
                                     c_vp(_ptr(W_out)), ctypes.byref(ns), c_vp(_stream(stream))))
    return ns.value


def gasa_power_estimate(n_units, bs, row_ptr, col, val, Dinv, x0, q, stream=None):
    rho = c_dbl()
    _check(load().gasa_power_estimate(c_i32(n_units), c_i32(bs), c_vp(_ptr(row_ptr)),
                                      c_vp(_ptr(col)), c_vp(_ptr(val)), c_vp(_ptr(Dinv)),
                                      c_vp(_ptr(x0)), c_i32(q), ctypes.byref(rho),
                                      c_vp(_stream(stream))))
    return rho.value


def gasa_power_estimate_noalloc(n_units, bs, row_ptr, col, val, Dinv, x0, q, stream=None):
    """gasa_power_estimate without any device allocation: the scratch is a
    fixed array inside the library (n_units * bs <= GASA_NOALLOC_MAX_DOFS),
    for callers that must not allocate when they run this step."""
    rho = c_dbl()
    _check(load().gasa_power_estimate_noalloc(c_i32(n_units), c_i32(bs), c_vp(_ptr(row_ptr)),
                                              c_vp(_ptr(col)), c_vp(_ptr(val)), c_vp(_ptr(Dinv)),
                                              c_vp(_ptr(x0)), c_i32(q), ctypes.byref(rho),
                                              c_vp(_stream(stream))))
    return rho.value


def gasa_relax_candidates(n_units, bs, row_ptr, col, val, W, B, r, gamma, max_relax,
                          stream=None):
    sw = (c_i32 * r)()
    _check(load().gasa_relax_candidates(c_i32(n_units), c_i32(bs), c_vp(_ptr(row_ptr)),
                                        c_vp(_ptr(col)), c_vp(_ptr(val)), c_vp(_ptr(W)),
                                        c_vp(_ptr(B)), c_i32(r), c_dbl(gamma), c_i32(max_relax),
                                        sw, c_vp(_stream(stream))))
    return np.array(sw[:], dtype=np.int32)


def gasa_tentative(n_units, bs, n_agg, agg_of, B, r, s_next, T_out, sigma_out=None, stream=None):
    return _check(load().gasa_tentative(c_i32(n_units), c_i32(bs), c_i32(n_agg),
                                        c_vp(_ptr(agg_of)), c_vp(_ptr(B)), c_i32(r),
                                        c_i32(s_next), c_vp(_ptr(T_out)), c_vp(_ptr(sigma_out)),
                                        c_vp(_stream(stream))))


def gasa_dense_inverse(n, A, Ainv, stream=None):
    sing = c_i32()
    _check(load().gasa_dense_inverse(c_i32(n), c_vp(_ptr(A)), c_vp(_ptr(Ainv)),
                                     ctypes.byref(sing), c_vp(_stream(stream))))
    return sing.value
