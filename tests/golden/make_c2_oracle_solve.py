"""Writes c2_oracle_solve.json: the oracle's own solves of the 1.31M-dof
P3 SIPG workload (256 x 256 jittered squares, 2 triangles each, r = 4,
levels by the paper's rule) to 1e-10 relative residual from x = 0.

For each precision (FP64 V-cycle in CG; float32 V-cycle in flexible CG) it
records the iteration count, the true relative residual, the 2-norm and
the max-norm of x, and x at 4,096 fixed sampled dofs, so that GPU tests can
compare their own solves with the oracle's without rerunning it (one oracle
solve takes about half an hour on one core).

Calls only the oracle and the seeded input recipe:
    python tests/golden/make_c2_oracle_solve.py [fp64|mixed32 ...] [--save-x DIR]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import gasa_oracle as O  # noqa: E402
from synth import configs  # noqa: E402

OUT = os.path.join(HERE, "c2_oracle_solve.json")
TOL = 1e-10
N_SAMPLES = 4096
SAMPLE_SEED = 2504


def sample_indices(n):
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, N_SAMPLES, replace=False))


def main(argv):
    precisions = [a for a in argv if not a.startswith("--") and a in ("fp64", "mixed32", "mixed16")]
    precisions = precisions or ["fp64", "mixed32"]
    save_dir = argv[argv.index("--save-x") + 1] if "--save-x" in argv else None
    pr = configs.poisson2d_p3()
    A = pr.A
    t0 = time.perf_counter()
    H = O.setup(A.row_ptr, A.col, A.val, pr.agg_of, B0=pr.B0, r=pr.r, dim=2)
    t_setup = time.perf_counter() - t0
    idx = sample_indices(pr.n_dofs)
    common = {
        "_about": ("Oracle solves of poisson2d_p3_256x256 (SIPG P3, penalty 90/h, r = 4, "
                   "levels L0..L8) to 1e-10 relative residual from x = 0, written by "
                   "make_c2_oracle_solve.py (oracle and seeded inputs only)."),
        "workload": pr.name, "dofs": int(pr.n_dofs), "tol": TOL,
        "level_dofs": [int(L.n) for L in H.levels],
        "sample_seed": SAMPLE_SEED, "sample_index": idx.tolist(),
        "setup_s": t_setup,
    }
    for prec in precisions:
        t0 = time.perf_counter()
        res = O.solve(H, pr.rhs, TOL, "cg", precision=prec, max_iter=10000)
        dt = time.perf_counter() - t0
        x = res.x
        rec = {"iterations": int(res.iterations), "converged": bool(res.converged),
               "rel_residual": float(res.rel_residual), "x_norm2": float(np.linalg.norm(x)),
               "x_norm_inf": float(np.max(np.abs(x))), "x_sample": x[idx].tolist(),
               "solve_s": dt}
        if save_dir:
            np.save(os.path.join(save_dir, f"c2_oracle_x_{prec}.npy"), x)
        # re-read before writing: runs of other precisions may share the file
        out = json.load(open(OUT)) if os.path.exists(OUT) else {}
        out.update(common)
        out[prec] = rec
        tmp = f"{OUT}.{prec}.tmp"
        with open(tmp, "w") as f:
            json.dump(out, f)
        os.replace(tmp, OUT)
        print(prec, res.iterations, res.rel_residual, f"{dt:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
