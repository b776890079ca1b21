"""Seeded random operands for single-operation parity tests (input recipe).

Random BSR patterns (sorted columns, optional diagonal), random dense blocks,
vectors and aggregate maps, all from splitmix64 streams >= 100 so they never
collide with the workload streams.  No arithmetic of the method lives here.
"""
import numpy as np

from . import rng


def random_bsr(n_rows: int, n_cols: int, br: int, bc: int, per_row: int, seed: int,
               diag: bool = False, stream: int = 100):
    """Each block row gets up to `per_row` distinct random block columns
    (plus the diagonal when `diag`); values uniform(-1, 1)."""
    u = rng.uniform(seed, stream, n_rows * per_row)
    cols = (u * n_cols).astype(np.int64).reshape(n_rows, per_row)
    rows = []
    for i in range(n_rows):
        c = set(cols[i].tolist())
        if diag:
            c.add(i)
        rows.append(sorted(c))
    ptr = np.zeros(n_rows + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(c) for c in rows])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    val = 2.0 * rng.uniform(seed, stream + 1, col.size * br * bc).reshape(-1, br, bc) - 1.0
    return ptr, col, val


def diagonally_dominant(ptr, col, val, shift: float = 4.0):
    """Add shift * (row count) to the diagonal entries of diagonal blocks so
    that block Jacobi inverses exist and are well conditioned."""
    val = val.copy()
    n = ptr.size - 1
    b = val.shape[1]
    for i in range(n):
        for k in range(ptr[i], ptr[i + 1]):
            if col[k] == i:
                val[k] += shift * (ptr[i + 1] - ptr[i]) * np.eye(b)
    return val


def random_vector(n: int, seed: int, stream: int = 110) -> np.ndarray:
    return 2.0 * rng.uniform(seed, stream, n) - 1.0


def random_normal(n: int, seed: int, stream: int = 111) -> np.ndarray:
    return rng.normal(seed, stream, n)


def random_blocks(m: int, b: int, seed: int, stream: int = 112) -> np.ndarray:
    return (2.0 * rng.uniform(seed, stream, m * b * b) - 1.0).reshape(m, b, b)


def chunk_aggregates(n_units: int, size: int) -> np.ndarray:
    """Consecutive units grouped `size` at a time (last group ragged)."""
    return (np.arange(n_units) // size).astype(np.int32)
