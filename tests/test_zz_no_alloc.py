"""The allocation-free power estimate against the allocating one.

gasa_power_estimate_noalloc serves callers that cannot allocate device
memory when they run this step (a fixed device-memory budget after
start-up, an allocator owned by a host framework, serving code that must
not block on or fail in the allocator); it keeps its scratch in a fixed
array inside the library.  This file sorts last so that a run stopping at
its first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import gasa_oracle as O
from synth import random_ops as RO
from tests.helpers import problem, to_dev

pytestmark = pytest.mark.gpu


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
    return A, dev


def test_noalloc_matches_allocating_entry_point_twice():
    """Two calls in a row (different matrices and start vectors, so the
    second call must not see the first call's scratch) agree with
    gasa_power_estimate to 1e-12 relative, the bar of the FP64 kernels."""
    gasa = _gasa()
    for name, seed in (("c1", 61), ("p3_16", 62)):
        A, d = _inputs(name)
        x0 = to_dev(RO.random_vector(A.n * A.b, seed))
        want = gasa.gasa_power_estimate(A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
        got = gasa.gasa_power_estimate_noalloc(A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
        assert abs(got - want) <= 1e-12 * want, (name, got, want)
        again = gasa.gasa_power_estimate_noalloc(A.n, A.b, d["rp"], d["col"], d["val"], d["Dinv"], x0, 3)
        assert again == got


def test_noalloc_rejects_sizes_beyond_the_scratch():
    gasa = _gasa()
    L = gasa.load()
    import ctypes
    n_units = gasa.GASA_NOALLOC_MAX_DOFS // 4 + 1       # 4-dof units, one unit too many
    rho = ctypes.c_double(-1.0)
    dummy = ctypes.c_void_p(16)                           # never dereferenced: rejected on the host
    st = L.gasa_power_estimate_noalloc(n_units, 4, dummy, dummy, dummy, dummy, dummy, 3,
                                       ctypes.byref(rho), None)
    assert st == gasa.GASA_ERR_INVALID_ARG
    assert rho.value == -1.0
