"""The allocation-free power estimate against the allocating one and the
oracle, and a check that it allocates nothing.

gasa_power_estimate_noalloc serves callers that cannot allocate device
memory when they run this step (a fixed device-memory budget after
start-up, an allocator owned by a host framework, serving code that must
not block on or fail in the allocator); it keeps its scratch in a fixed
array inside the library.  This file sorts last so that a run stopping at
its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import gasa_oracle as O
from synth import random_ops as RO
from tests.helpers import problem, to_dev

pytestmark = pytest.mark.gpu

MEMPOOL_ATTR_RESERVED_MEM_CURRENT = 0x5
MEMPOOL_ATTR_USED_MEM_CURRENT = 0x7
MEMPOOL_ATTR_USED_MEM_HIGH = 0x8


def _gasa():
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    return gasa


def _inputs(name):
    A = problem(name).A
    up = np.arange(A.n + 1) * A.b
    Dinv = O.invert_blocks(O.block_diagonal(A.to_scipy(), up))
    dev = dict(rp=to_dev(A.row_ptr), col=to_dev(A.col), val=to_dev(A.val.ravel()),
               Dinv=to_dev(Dinv.blocks.ravel()))
    return A, Dinv, dev


def _pool(rt, device=0):
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), device) == 0
    return pool


def _pool_attr(rt, pool, attr):
    v = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


def _reset_used_high(rt, pool):
    zero = ctypes.c_uint64(0)           # the watermark can only be reset, to zero
    assert rt.cudaMemPoolSetAttribute(pool, MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _memory_state(device=0):
    """(free device bytes, default pool reserved bytes, default pool used
    bytes), read through the CUDA runtime the library itself links."""
    rt = ctypes.CDLL("libcudart.so.13")
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    pool = _pool(rt, device)
    return (free.value, _pool_attr(rt, pool, MEMPOOL_ATTR_RESERVED_MEM_CURRENT),
            _pool_attr(rt, pool, MEMPOOL_ATTR_USED_MEM_CURRENT))


def test_noalloc_matches_allocating_entry_point_and_oracle_twice():
    """Two calls in a row (different matrices and start vectors, so the
    second call must not see the first call's scratch) agree with
    gasa_power_estimate and with the oracle's Alg. 4 to 1e-12 relative, the
    bar of the FP64 kernels; a repeated call gives the same bits."""
    gasa = _gasa()
    for name, seed in (("c1", 61), ("p3_16", 62)):
        A, Dinv, d = _inputs(name)
        x0h = RO.random_vector(A.n * A.b, seed)
        x0 = to_dev(x0h)
        want = gasa.gasa_power_estimate(A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
        got = gasa.gasa_power_estimate_noalloc(A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
        oracle = O.power_estimate(A.to_scipy(), Dinv, x0h / np.linalg.norm(x0h), 3)
        assert abs(got - want) <= 1e-12 * want, (name, got, want)
        assert abs(got - oracle) <= 1e-12 * oracle, (name, got, oracle)
        again = gasa.gasa_power_estimate_noalloc(A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
        assert again == got


def test_noalloc_allocates_no_device_memory():
    """After a first call, further calls leave the device's free memory and
    the default memory pool's reserved and used bytes unchanged, and the
    pool's high watermark of used bytes, reset before the calls, shows no
    allocation inside them either.  The watermark does rise for the
    allocating entry point (its scratch comes from the default pool), so it
    is able to see an allocation."""
    import torch
    gasa = _gasa()
    rt = ctypes.CDLL("libcudart.so.13")
    pool = _pool(rt)
    A, _, d = _inputs("p3_16")
    x0 = to_dev(RO.random_vector(A.n * A.b, 63))
    args = (A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
    gasa.gasa_power_estimate_noalloc(*args)          # first call: module and symbol set up
    torch.cuda.synchronize()
    before = _memory_state()
    _reset_used_high(rt, pool)
    for _ in range(3):
        gasa.gasa_power_estimate_noalloc(*args)
    torch.cuda.synchronize()
    assert _memory_state() == before
    assert _pool_attr(rt, pool, MEMPOOL_ATTR_USED_MEM_HIGH) <= before[2]
    # positive control: the allocating variant's scratch shows in the watermark
    _reset_used_high(rt, pool)
    gasa.gasa_power_estimate(*args)
    torch.cuda.synchronize()
    n = A.n * A.b
    assert _pool_attr(rt, pool, MEMPOOL_ATTR_USED_MEM_HIGH) >= 2 * n * 8


def test_noalloc_rejects_sizes_beyond_the_scratch():
    gasa = _gasa()
    L = gasa.load()
    n_units = gasa.GASA_NOALLOC_MAX_DOFS // 4 + 1       # 4-dof units, one unit too many
    rho = ctypes.c_double(-1.0)
    dummy = ctypes.c_void_p(16)                           # never dereferenced: rejected on the host
    st = L.gasa_power_estimate_noalloc(n_units, 4, dummy, dummy, dummy, dummy, dummy, 3,
                                       ctypes.byref(rho), None)
    assert st == gasa.GASA_ERR_INVALID_ARG
    assert rho.value == -1.0
