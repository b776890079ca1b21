"""The oracle against the iteration table the paper prints for its
structured Poisson example (Section 6.1): Q1 hexahedra on [-1, 1]^3, 2^M per
side, interior penalty and minimal-dissipation LDG fluxes, Dirichlet on
x = -1, Neumann elsewhere, the manufactured right-hand side, tolerance 1e-7
from a zero initial guess, three pre- and post-smoothing steps.

The paper's aggregates come from METIS; these come from recursive coordinate
bisection, which on this Cartesian mesh gives exact 2x2x2 aggregates at every
level.  So the counts are compared as a band, not for parity: the pCG count
within one of the paper's, and the stationary count no lower than the
paper's and at most three above it (the stationary solver is the more
sensitive of the two to the hierarchy's last level, which here keeps 136
dofs at M = 4 where the paper's keeps 100).  The pCG count must also stay
flat under refinement (near mesh independence, the paper's abstract).
M = 5 (262,144 dofs) takes minutes on one core; it runs when the
environment variable GASA_SLOW_ORACLE is set."""
import functools
import json
import os

import numpy as np
import pytest

from oracle import gasa_oracle as O
from synth import configs

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = json.load(open(os.path.join(HERE, "golden", "paper_hex_table.json")))


@functools.lru_cache(maxsize=None)
def _counts(M, flux):
    pr = configs.poisson3d_hex(M, flux=flux)
    A = pr.A
    H = O.setup(A.row_ptr, A.col, A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=3)
    tol = TABLE["tol"]
    cg = O.solve(H, pr.rhs, tol, "cg", max_iter=200)
    st = O.stationary(H, pr.rhs, tol, max_iter=200)
    assert cg.converged and st.converged
    return cg.iterations, st.iterations, [L.n for L in H.levels]


def _check(M, flux):
    cg, st, _ = _counts(M, flux)
    paper_cg = TABLE[flux]["pcg"][str(M)]
    paper_st = TABLE[flux]["stationary"][str(M)]
    assert abs(cg - paper_cg) <= 1, (flux, M, cg, paper_cg)
    assert paper_st <= st <= paper_st + 3, (flux, M, st, paper_st)


@pytest.mark.parametrize("flux", ["ip", "ldg"])
@pytest.mark.parametrize("M", [3, 4])
def test_hex_iteration_counts_in_the_papers_band(M, flux):
    _check(M, flux)


@pytest.mark.parametrize("flux", ["ip", "ldg"])
def test_hex_pcg_counts_flat_under_refinement(flux):
    assert _counts(4, flux)[0] - _counts(3, flux)[0] <= 1


def test_hex_hierarchy_sizes_against_the_papers():
    """Level sizes at M = 4 (IP): the top two equal the paper's up to the
    aggregates' shape (5,120 vs 5,206: METIS splits unevenly, RCB evenly);
    level 3 keeps 17 vectors per aggregate here and 100 / 8 = 12.5 in the
    paper, a count Eq. sik does not produce (parity unpinned there)."""
    sizes = _counts(4, "ip")[2]
    paper = TABLE["hierarchy_M4_ip_dofs"]["value"]
    assert sizes[0] == paper[0]
    assert sizes[1:] == [512 * (64 // 6), 64 * ((8 * (64 // 6)) // 6), 8 * ((8 * 13) // 6)]
    for ours, theirs in zip(sizes[1:3], paper[1:3]):
        assert abs(ours - theirs) <= 0.06 * theirs


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("GASA_SLOW_ORACLE"), reason="M = 5 takes minutes on one core")
@pytest.mark.parametrize("flux", ["ip", "ldg"])
def test_hex_iteration_counts_M5(flux):
    _check(5, flux)
