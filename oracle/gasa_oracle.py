"""CPU reference (oracle) for geometric adaptive smoothed aggregation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module; the library never
does, and this module imports nothing from the library.

Plain, slow, FP64 numpy/scipy restatement of the method of Pan, Lindsey &
Persson, "Geometric adaptive smoothed aggregation multigrid for
discontinuous Galerkin discretisations" (2025), written step by step in the
paper's order.  Library primitives (sparse products, dense inverse, SVD)
serve as single steps; nothing is blocked, fused or reordered.

Naming: the paper writes the tentative (orthonormal, block-diagonal)
prolongator as P_{k+1}^k and the smoothed one as T_{k+1}^k = S_k P.  This
code calls the tentative one T and the smoothed one P = (I - w D^-1 A) T,
with R = P^T.

Readings where the paper is silent or garbled (each listed in the design
notes as well):
* the relaxation stop test of Eq. bsmooth compares the last two iterates,
  so at least one sweep runs, the sweep that satisfies the test is kept and
  at most `max_relax` sweeps run;
* Eq. sik (h-branch) s_j = |A_j| / n_cut is read as
  min(max(1, floor(rows_j / n_cut)), r, rows_j);
* left singular vectors are ordered by descending singular value and each
  kept column is signed so that its entry of largest magnitude (lowest row
  on ties) is positive;
* a kept singular value at or below 1e-10 sigma_1 counts as zero (the
  candidate block has lower numerical rank than the kept count); its vector
  is replaced by the Gram-Schmidt completion of unit vectors described in
  `complete_null_columns`;
* Alg. 2's post-smoothing right-hand side is the level right-hand side b_k;
* Alg. 4's start vector is uniform(-1, 1) per entry from splitmix64 stream
  4 + 16 k (level k), normalised;
* B^{k+1} = R B^k (Alg. 5), with T^T B^k (Eq. SA_Bk) as an option.

Mixed precision (not in the paper): the V-cycle runs in float32 (float32
operators, float32 vectors and accumulation), the coarsest dense solve in
float64, inside float64 flexible CG or FGMRES.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

GOLDEN = 0x9E3779B97F4A7C15
MASK = 0xFFFFFFFFFFFFFFFF


# ----------------------------------------------------------------------------
# splitmix64 (Steele, Lea & Flood 2014), written out independently here
# ----------------------------------------------------------------------------

def splitmix_uniform(seed: int, stream: int, n: int) -> np.ndarray:
    key = np.uint64((seed & MASK) ^ ((stream * GOLDEN) & MASK))
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def power_start_vector(seed: int, level: int, n: int) -> np.ndarray:
    """Alg. 4 line 1: a random vector of unit norm (uniform(-1,1) entries)."""
    x = 2.0 * splitmix_uniform(seed, 4 + 16 * level, n) - 1.0
    return x / np.linalg.norm(x)


# ----------------------------------------------------------------------------
# block-diagonal operators on a level (units = elements or aggregates)
# ----------------------------------------------------------------------------

class BlockDiag:
    """Dense blocks on the diagonal, one per unit; unit u owns dofs
    unit_ptr[u] .. unit_ptr[u+1]-1.  Equal-sized blocks are kept stacked."""

    def __init__(self, unit_ptr, blocks):
        self.unit_ptr = np.asarray(unit_ptr, np.int64)
        sizes = np.diff(self.unit_ptr)
        self.uniform = sizes.size > 0 and np.all(sizes == sizes[0])
        if self.uniform and not isinstance(blocks, np.ndarray):
            blocks = np.stack(blocks) if len(blocks) else np.zeros((0, 0, 0))
        if not self.uniform and isinstance(blocks, np.ndarray):
            blocks = list(blocks)
        self.blocks = blocks

    def apply(self, x: np.ndarray) -> np.ndarray:
        if self.uniform:
            s = self.blocks.shape[1]
            return np.einsum("uij,uj->ui", self.blocks, x.reshape(-1, s)).ravel()
        y = np.empty_like(x)
        up = self.unit_ptr
        for u, Bk in enumerate(self.blocks):
            y[up[u]:up[u + 1]] = Bk @ x[up[u]:up[u + 1]]
        return y

    def to_sparse(self) -> sp.csr_matrix:
        if self.uniform:
            m = self.blocks.shape[0]
            return sp.bsr_matrix((self.blocks, np.arange(m), np.arange(m + 1)),
                                 shape=(self.unit_ptr[-1],) * 2).tocsr()
        return sp.block_diag(self.blocks, format="csr")

    def scaled(self, w):
        if self.uniform:
            return BlockDiag(self.unit_ptr, w * self.blocks)
        return BlockDiag(self.unit_ptr, [w * b for b in self.blocks])

    def astype(self, dt):
        if self.uniform:
            return BlockDiag(self.unit_ptr, self.blocks.astype(dt))
        return BlockDiag(self.unit_ptr, [b.astype(dt) for b in self.blocks])


def block_diagonal(A: sp.csr_matrix, unit_ptr: np.ndarray) -> BlockDiag:
    """D_k: the diagonal blocks of A_k, one per unit (Eq. smoother_choice,
    block Jacobi P(A_k) = D_k)."""
    A = A.tocsr()
    unit_ptr = np.asarray(unit_ptr, np.int64)
    sizes = np.diff(unit_ptr)
    if sizes.size and np.all(sizes == sizes[0]):
        s = int(sizes[0])
        Ab = A.tobsr(blocksize=(s, s))
        Ab.sort_indices()
        m = sizes.size
        out = np.zeros((m, s, s))
        rows = np.repeat(np.arange(m), np.diff(Ab.indptr))
        on_diag = Ab.indices == rows
        out[rows[on_diag]] = Ab.data[on_diag]
        return BlockDiag(unit_ptr, out)
    blocks = []
    for u in range(unit_ptr.size - 1):
        a, b = unit_ptr[u], unit_ptr[u + 1]
        blocks.append(A[a:b, a:b].toarray())
    return BlockDiag(unit_ptr, blocks)


def invert_blocks(D: BlockDiag) -> BlockDiag:
    if D.uniform:
        return BlockDiag(D.unit_ptr, np.linalg.inv(D.blocks))
    return BlockDiag(D.unit_ptr, [np.linalg.inv(b) for b in D.blocks])


# ----------------------------------------------------------------------------
# Alg. 1 (Smooth) and the block Jacobi smoother
# ----------------------------------------------------------------------------

def smooth_step(x, A, W: BlockDiag, b):
    """One step of Alg. 1: x <- x + A~^{-1} (b - A x), A~^{-1} = w D^{-1}."""
    return x + W.apply(b - A @ x)


def smooth_fixed(u0, A, W, b, t):
    """Alg. 1 with stop(.) = (m >= t)."""
    x = u0
    for _ in range(t):
        x = smooth_step(x, A, W, b)
    return x


# ----------------------------------------------------------------------------
# Alg. 4 and Eq. omega
# ----------------------------------------------------------------------------

def power_estimate(A, Dinv: BlockDiag, x0, q: int = 3) -> float:
    """Alg. 4: q times x <- A x; x <- P^{-1} x; x <- x / ||x||; then return
    ||P^{-1} A x||."""
    x = x0.copy()
    for _ in range(q):
        x = A @ x
        x = Dinv.apply(x)
        x = x / np.linalg.norm(x)
    return float(np.linalg.norm(Dinv.apply(A @ x)))


def omega_from_rho(rho: float, factor: float = 4.0 / 3.0) -> float:
    """Eq. omega: w_k = (4/3) / rho_k."""
    return factor / rho


# ----------------------------------------------------------------------------
# Eq. bsmooth: adaptive relaxation of candidates on A x = 0
# ----------------------------------------------------------------------------

def relax_candidates(A, W: BlockDiag, B: np.ndarray, gamma: float = 0.03, max_relax: int = 100):
    """Each column: x^(m) = x^(m-1) + W (0 - A x^(m-1)) until
    ||x^(m-1)|| / ||x^(m)|| < 1 + gamma.  Returns (B relaxed, sweeps)."""
    B = np.array(B, dtype=np.float64, order="F", copy=True)
    sweeps = np.zeros(B.shape[1], dtype=np.int32)
    zero = np.zeros(B.shape[0])
    for j in range(B.shape[1]):
        x = B[:, j].copy()
        nx = np.linalg.norm(x)
        m = 0
        while m < max_relax:
            x_new = smooth_step(x, A, W, zero)
            m += 1
            n_new = np.linalg.norm(x_new)
            x = x_new
            if nx / n_new < 1.0 + gamma:
                break
            nx = n_new
        B[:, j] = x
        sweeps[j] = m
    return B, sweeps


# ----------------------------------------------------------------------------
# Eq. splitB_dg + Eq. sik: tentative prolongator by per-aggregate SVD
# ----------------------------------------------------------------------------

def keep_count(rows: int, r: int, n_cut: float) -> int:
    """Eq. sik, h-multigrid branch: |A_j| / n_cut, floored, at least 1, at
    most the r candidates and the rows of the block."""
    return int(min(max(1, int(np.floor(rows / n_cut))), r, rows))


def hstar_keep(S: np.ndarray, delta: float) -> int:
    """Eq. sik, h*-multigrid branch (an aggregate that is one element of the
    level above): the number of singular values above delta * sigma_1."""
    return max(1, int(np.count_nonzero(S > delta * S[0])))


NULL_SIGMA = 1e-10


def complete_null_columns(U: np.ndarray, S: np.ndarray, s: int) -> np.ndarray:
    """Kept columns whose singular value is numerically zero
    (sigma_l <= NULL_SIGMA * sigma_1) carry no information from the
    candidates; they are replaced, in order, by unit vectors e_t
    (t = l, l+1, ... cyclically) orthogonalised twice against the columns
    already fixed, the first with norm above 1/2 being kept."""
    rows = U.shape[0]
    U = U[:, :s].copy()
    smax = S[0] if S.size else 0.0
    for l in range(s):
        if l < S.size and S[l] > NULL_SIGMA * smax:
            continue
        for t in range(rows):
            v = np.zeros(rows)
            v[(l + t) % rows] = 1.0
            for _ in range(2):
                for m in range(l):
                    v = v - (U[:, m] @ v) * U[:, m]
            nv = np.linalg.norm(v)
            if nv * nv > 0.25:
                U[:, l] = v / nv
                break
    return U


def sign_fix(U: np.ndarray) -> np.ndarray:
    U = U.copy()
    for c in range(U.shape[1]):
        m = int(np.argmax(np.abs(U[:, c])))
        if U[m, c] < 0:
            U[:, c] = -U[:, c]
    return U


def aggregate_rows(agg: np.ndarray, unit_ptr: np.ndarray, n_agg: int):
    """Dofs of every aggregate: children in increasing unit id, each unit's
    dofs in order."""
    rows = [[] for _ in range(n_agg)]
    for u in range(agg.size):
        rows[agg[u]].extend(range(unit_ptr[u], unit_ptr[u + 1]))
    return [np.array(rw, dtype=np.int64) for rw in rows]


def tentative(B: np.ndarray, agg: np.ndarray, unit_ptr: np.ndarray, n_agg: int,
              n_cut: float, keep: Optional[List[int]] = None, delta: Optional[float] = None):
    """T = blockdiag(U_j[:, :s_j]) with B[A_j, :] = U_j S_j V_j^T; s_j by the
    h-branch of Eq. sik, or by its h*-branch when delta is given.
    Returns (T as csr, next-level unit_ptr, singular values per aggregate)."""
    r = B.shape[1]
    rows = aggregate_rows(agg, unit_ptr, n_agg)
    cols_ptr = np.zeros(n_agg + 1, dtype=np.int64)
    Us, svals = [], []
    for J in range(n_agg):
        BJ = B[rows[J], :]
        U, S, _ = np.linalg.svd(BJ, full_matrices=False)
        if keep is not None:
            s = keep[J]
        elif delta is not None:
            s = hstar_keep(S, delta)
        else:
            s = keep_count(len(rows[J]), r, n_cut)
        Us.append(sign_fix(complete_null_columns(U, S, s)))
        svals.append(S)
        cols_ptr[J + 1] = cols_ptr[J] + s
    n_rows = unit_ptr[-1]
    ri, ci, vv = [], [], []
    for J in range(n_agg):
        rr, cc = np.meshgrid(rows[J], np.arange(cols_ptr[J], cols_ptr[J + 1]), indexing="ij")
        ri.append(rr.ravel())
        ci.append(cc.ravel())
        vv.append(Us[J].ravel())
    T = sp.csr_matrix((np.concatenate(vv), (np.concatenate(ri), np.concatenate(ci))),
                      shape=(n_rows, cols_ptr[-1]))
    return T, cols_ptr, svals


# ----------------------------------------------------------------------------
# Eq. TR0, Eq. SA_restrict, Galerkin product, candidate transfer
# ----------------------------------------------------------------------------

def smoothed_prolongator(A, W: BlockDiag, T):
    """P = (I - w D^{-1} A) T = T - W (A T)."""
    return (T - W.to_sparse() @ (A @ T)).tocsr()


def galerkin(R, A, P):
    """A_{k+1} = R A_k P."""
    return (R @ (A @ P)).tocsr()


# ----------------------------------------------------------------------------
# structural block patterns (no numerical dropping)
# ----------------------------------------------------------------------------

def pattern_csr(pat: sp.csr_matrix):
    pat = pat.tocsr()
    pat.sort_indices()
    return pat.indptr.astype(np.int64), pat.indices.astype(np.int64)


def bool_csr(ptr, idx, shape):
    return sp.csr_matrix((np.ones(idx.size), idx, ptr), shape=shape)


def aggregation_matrix(agg, n_agg):
    n = agg.size
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, n_agg))


# ----------------------------------------------------------------------------
# setup: Alg. 5
# ----------------------------------------------------------------------------

@dataclass
class Level:
    A: sp.csr_matrix
    unit_ptr: np.ndarray
    Apat: sp.csr_matrix                 # block pattern of A_k (units x units)
    W: Optional[BlockDiag] = None       # w_k D_k^{-1}
    Dinv: Optional[BlockDiag] = None
    rho: float = 0.0
    omega: float = 0.0
    B_in: Optional[np.ndarray] = None   # candidates before relaxation
    B: Optional[np.ndarray] = None      # relaxed candidates
    sweeps: Optional[np.ndarray] = None
    T: Optional[sp.csr_matrix] = None
    P: Optional[sp.csr_matrix] = None
    R: Optional[sp.csr_matrix] = None
    Ppat: Optional[sp.csr_matrix] = None
    svals: Optional[list] = None

    @property
    def n(self):
        return self.A.shape[0]


@dataclass
class Hierarchy:
    levels: List[Level]
    coarse: np.ndarray                  # dense A_N
    t_pre: int = 3
    t_post: int = 3
    r: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return len(self.levels) - 1


def bsr_to_csr(row_ptr, col, val):
    n = row_ptr.size - 1
    b = val.shape[1]
    return sp.bsr_matrix((val, col, row_ptr), shape=(n * b, n * b)).tocsr()


def median_aggregate_dofs(agg1, unit_ptr0, n_agg1):
    """Section 4.2: r = median dof count of a level-1 aggregate (the lower
    median for an even count)."""
    sizes = np.zeros(n_agg1, dtype=np.int64)
    np.add.at(sizes, agg1, np.diff(unit_ptr0))
    s = np.sort(sizes)
    return int(s[(s.size - 1) // 2])


def setup(row_ptr, col, val, agg_of, B0=None, r=None, dim=2, seed=13373,
          gamma=0.03, q=3, omega_factor=4.0 / 3.0, n_cut=None, max_relax=100,
          t_pre=3, t_post=3, cand_init="R", hstar=False, delta=1e-3):
    """Alg. 5 with the hierarchy given (levels L0..LN, N = len(agg_of)).
    hstar: one h*-multigrid step at the top (Section 4.3): level 0 and its
    elements are duplicated (every element its own aggregate) and the kept
    count follows the h*-branch of Eq. sik with threshold delta; the given
    hierarchy follows, one level lower.  r still comes from the first
    geometric aggregates."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    nb = val.shape[1]
    n_units = row_ptr.size - 1
    if n_cut is None:
        n_cut = 2 ** dim - (dim - 1)
    A = bsr_to_csr(row_ptr, col, val)
    unit_ptr = np.arange(n_units + 1, dtype=np.int64) * nb
    Apat = bool_csr(row_ptr, col, (n_units, n_units))
    levels = [Level(A, unit_ptr, Apat)]
    n_agg1 = int(agg_of[0].max()) + 1 if agg_of else 1
    if r is None or r == 0:
        r = median_aggregate_dofs(agg_of[0], unit_ptr, n_agg1)
    if B0 is None:
        raise ValueError("the oracle takes B^0 as an input")
    B = np.array(B0, dtype=np.float64, order="F")[:, :r]
    if hstar:
        agg_of = [np.arange(n_units)] + list(agg_of)
    for k, agg in enumerate(agg_of):
        L = levels[k]
        agg = np.asarray(agg, np.int64)
        n_agg = int(agg.max()) + 1
        # smoother: Alg. 4 + Eq. omega + Eq. smoother_choice
        L.Dinv = invert_blocks(block_diagonal(L.A, L.unit_ptr))
        L.rho = power_estimate(L.A, L.Dinv, power_start_vector(seed, k, L.n), q)
        L.omega = omega_from_rho(L.rho, omega_factor)
        L.W = L.Dinv.scaled(L.omega)
        # Eq. bsmooth
        L.B_in = B
        L.B, L.sweeps = relax_candidates(L.A, L.W, B, gamma, max_relax)
        # Eq. splitB_dg + Eq. sik
        L.T, next_ptr, L.svals = tentative(L.B, agg, L.unit_ptr, n_agg, n_cut,
                                           delta=delta if (hstar and k == 0) else None)
        # Eq. TR0 and Eq. SA_restrict
        L.P = smoothed_prolongator(L.A, L.W, L.T)
        L.R = L.P.T.tocsr()
        G = aggregation_matrix(agg, n_agg)
        L.Ppat = ((L.Apat @ G) != 0).astype(np.float64).tocsr()
        APpat = ((L.Apat @ L.Ppat) != 0).astype(np.float64)
        Anext_pat = ((L.Ppat.T @ APpat) != 0).astype(np.float64).tocsr()
        # Galerkin operator and next candidates (Alg. 5)
        A_next = galerkin(L.R, L.A, L.P)
        if cand_init == "R":
            B = np.asfortranarray(L.R @ L.B)
        else:
            B = np.asfortranarray(L.T.T @ L.B)
        levels.append(Level(A_next, next_ptr, Anext_pat))
    coarse = levels[-1].A.toarray()
    return Hierarchy(levels, coarse, t_pre, t_post, r)


# ----------------------------------------------------------------------------
# Alg. 2: V-cycle (one pass from a zero initial guess), FP64 or float32
# ----------------------------------------------------------------------------

def fp16_blocks(blocks: np.ndarray) -> np.ndarray:
    """Dense blocks stored as FP16 values v / s with one scale s = max |v| per
    block (s = 1 for a zero block), returned dequantised in float32."""
    m = np.max(np.abs(blocks), axis=(1, 2))
    s = np.where(m > 0, m, 1.0).astype(np.float32)
    h = (blocks / s.astype(np.float64)[:, None, None]).astype(np.float16)
    return h.astype(np.float32) * s[:, None, None]


class GalerkinOperator:
    """A_k applied without storing it (Section 4.4, Eq. matfree2 with the
    multi-level transfers of Eq. matfree1 unrolled): A_k x = R_{k-1} (A_{k-1}
    (P_{k-1} x)), where A_{k-1} is itself stored or of this kind."""

    def __init__(self, R, A_prev, P):
        self.R, self.A_prev, self.P = R, A_prev, P

    def __matmul__(self, x):
        return self.R @ (self.A_prev @ (self.P @ x))


def make_vcycle(H: Hierarchy, precision: str = "fp64", matrix_free_levels: int = 0):
    """Returns a function f -> u approximating A^{-1} f by one V-cycle.
    precision: 'fp64', 'fp32' (float32 operators and vectors), or 'fp16'
    (as 'fp32', with the level-0 operator and block inverses stored as FP16
    blocks with one scale per block).  matrix_free_levels = kappa: the
    operators A_1 .. A_kappa (kappa < N) are applied through the transfers
    (Section 4.4) instead of being used as stored matrices; in 'fp16' the
    level-0 operator inside those products is the float32 one."""
    N = H.N
    if precision == "fp64":
        dt = np.float64
        As = [L.A for L in H.levels[:N]]
        Ws = [L.W for L in H.levels[:N]]
        Ps = [L.P for L in H.levels[:N]]
        Rs = [L.R for L in H.levels[:N]]
    else:
        dt = np.float32
        As = [L.A.astype(np.float32) for L in H.levels[:N]]
        Ws = [L.W.astype(np.float32) for L in H.levels[:N]]
        Ps = [L.P.astype(np.float32) for L in H.levels[:N]]
        Rs = [L.R.astype(np.float32) for L in H.levels[:N]]
        if precision == "fp16":
            L0 = H.levels[0]
            b = int(L0.unit_ptr[1] - L0.unit_ptr[0])
            Ab = L0.A.tobsr(blocksize=(b, b))
            Ab.sort_indices()
            As[0] = sp.bsr_matrix((fp16_blocks(Ab.data.astype(np.float64)), Ab.indices, Ab.indptr),
                                  shape=Ab.shape).tocsr()
            Ws[0] = BlockDiag(L0.unit_ptr, fp16_blocks(L0.W.blocks))
    if matrix_free_levels > 0:
        stored0 = As[0] if precision != "fp16" else H.levels[0].A.astype(np.float32)
        prev = stored0
        for k in range(1, min(matrix_free_levels, N - 1) + 1):
            prev = GalerkinOperator(Rs[k - 1], prev, Ps[k - 1])
            As[k] = prev
    coarse = H.coarse

    def vcycle(f):
        b = [None] * (N + 1)
        u = [None] * (N + 1)
        b[0] = np.asarray(f, dtype=dt)
        for k in range(N):
            u[k] = smooth_fixed(np.zeros_like(b[k]), As[k], Ws[k], b[k], H.t_pre)
            r = b[k] - As[k] @ u[k]
            b[k + 1] = Rs[k] @ r
        u[N] = np.linalg.solve(coarse, b[N].astype(np.float64)).astype(dt)
        for k in range(N - 1, -1, -1):
            u[k] = u[k] + Ps[k] @ u[k + 1]
            u[k] = smooth_fixed(u[k], As[k], Ws[k], b[k], H.t_post)
        return u[0].astype(np.float64)

    return vcycle


# ----------------------------------------------------------------------------
# outer Krylov solvers (FP64)
# ----------------------------------------------------------------------------

@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    rel_residual: float
    converged: bool
    history: list


def pcg(A, b, M, tol=1e-10, max_iter=500, flexible=False) -> SolveResult:
    """Preconditioned CG from x0 = 0; `flexible` uses the Polak-Ribiere
    beta = r_{k+1}^T (z_{k+1} - z_k) / (r_k^T z_k).  The recurrence residual
    triggers the stop; the true residual must confirm it."""
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = r @ z
    hist = []
    for it in range(1, max_iter + 1):
        q = A @ p
        pq = p @ q
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel <= tol:
            true_r = b - A @ x
            rel_t = np.linalg.norm(true_r) / bn
            if rel_t <= tol:
                return SolveResult(x, it, rel_t, True, hist)
            r = true_r
        z_new = M(r)
        rz_new = r @ z_new
        beta = (rz_new - r @ z) / rz if flexible else rz_new / rz
        z = z_new
        p = z + beta * p
        rz = rz_new
    return SolveResult(x, max_iter, np.linalg.norm(b - A @ x) / bn, False, hist)


def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0
    h = np.hypot(a, b)
    return a / h, b / h


def gmres(A, b, M, tol=1e-10, restart=30, max_iter=1000, flexible=False) -> SolveResult:
    """GMRES(restart) from x0 = 0 with modified Gram-Schmidt Arnoldi and
    Givens rotations.  Left-preconditioned (Arnoldi on M A) by default; with
    `flexible`, right-preconditioned FGMRES that stores z_j = M v_j.
    Iterations = preconditioner applications inside Arnoldi."""
    bn = np.linalg.norm(b)
    n = b.size
    x = np.zeros_like(b)
    total = 0
    hist = []
    inner_tol = None
    while total < max_iter:
        r = b - A @ x
        rel = np.linalg.norm(r) / bn
        if rel <= tol:
            return SolveResult(x, total, rel, True, hist)
        v0 = r if flexible else M(r)
        beta = np.linalg.norm(v0)
        if inner_tol is None:
            inner_tol = tol * (bn if flexible else beta)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n)) if flexible else None
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = v0 / beta
        j_done = 0
        for j in range(restart):
            if flexible:
                Z[j] = M(V[j])
                w = A @ Z[j]
            else:
                w = M(A @ V[j])
            total += 1
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j_done = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= inner_tol or total >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        if flexible:
            x = x + Z[:j_done].T @ y
        else:
            x = x + V[:j_done].T @ y
    rel = np.linalg.norm(b - A @ x) / bn
    return SolveResult(x, total, rel, rel <= tol, hist)


def solve(H: Hierarchy, b, tol=1e-10, solver="cg", precision="fp64", restart=30, max_iter=500,
          matrix_free_levels=0):
    """x = A_0^{-1} b by V-cycle-preconditioned CG or GMRES (FP64 outer loop;
    with precision='mixed32' the V-cycle is float32 and the outer loop is
    flexible)."""
    M = make_vcycle(H, {"fp64": "fp64", "mixed32": "fp32", "mixed16": "fp16"}[precision],
                    matrix_free_levels)
    flex = precision != "fp64"
    A = H.levels[0].A
    if solver == "cg":
        return pcg(A, b, M, tol, max_iter, flexible=flex)
    return gmres(A, b, M, tol, restart, max_iter, flexible=flex)


def stationary(H: Hierarchy, b, tol=1e-10, max_iter=200, precision="fp64") -> SolveResult:
    """Alg. 2 as a solver: x <- x + V(b - A x) until ||b - A x|| <= tol ||b||.
    With precision='mixed32' the V-cycle is float32 and the residual and
    update stay float64 (iterative refinement)."""
    M = make_vcycle(H, {"fp64": "fp64", "mixed32": "fp32", "mixed16": "fp16"}[precision])
    A = H.levels[0].A
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = []
    for it in range(1, max_iter + 1):
        x = x + M(b - A @ x)
        rel = np.linalg.norm(b - A @ x) / bn
        hist.append(rel)
        if rel <= tol:
            return SolveResult(x, it, rel, True, hist)
    return SolveResult(x, max_iter, hist[-1], False, hist)


# ----------------------------------------------------------------------------
# single kernels, for per-step parity
# ----------------------------------------------------------------------------

def bsr_matvec(row_ptr, col, val, x, n_cols_blocks=None):
    """y = A x for a BSR matrix with (br x bc) blocks."""
    n = row_ptr.size - 1
    br, bc = val.shape[1], val.shape[2]
    nc = n_cols_blocks if n_cols_blocks is not None else n
    A = sp.bsr_matrix((val, col, row_ptr), shape=(n * br, nc * bc))
    return A @ x


def dense_block_inverses(blocks: np.ndarray) -> np.ndarray:
    return np.linalg.inv(blocks)
