#!/usr/bin/env python
"""Solves/s of alpha-SA-preconditioned CG on the P3 SIPG Poisson workload.

Workload: unit square, 256 x 256 squares jittered +-0.2h, 2 triangles each,
SIPG P3 (131072 elements, 1,310,720 dofs, 10 x 10 blocks), candidates r = 4,
levels L0..L8 by the paper's rule, right-hand side N(0,1).  One step = one
solve to ||b - A x|| <= 1e-10 ||b|| from x = 0 on the resident hierarchy
(setup is timed separately).  The headline value is the mixed-precision
solve (FP32 V-cycle inside FP64 flexible CG); the FP64 V-cycle solve is
reported beside it.  Every matrix pass streams more than the 129 MB L2
(A: 419 MB FP64, 209 MB FP32), so no L2 flush is needed between steps.

Multi-GPU: the path does not shard; --gpus N runs N independent replicas
(one process per GPU under torchrun) and reports the total solves/s; the
serving stream (a per-GPU measurement) runs at N = 1 only.

--impl reference times the CPU oracle on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s to 1e-10 rel. resid: mixed vs FP64 V-cycle; HBM GB/s; p50/p99 ms"
TOL = 1e-10
WORKLOAD = "poisson2d_sipg_p3_tri_256x256"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per launch of the level-0 FP32 smoothing sweep
# from one ncu capture each, valid while the kernel's source file hashes to
# `src_sha`: the plain kernel and the bulk-copy staged one.
# kernel classes of gasa_profile_read, timed by CUDA events in the host-driven loop
PROFILE_CLASSES = ["level0_step", "level0_residual_restriction", "outer_Ap", "level0_first_step",
                   "level0_prolongation"]

NCU_TRAFFIC = {
    # captured on the 224x224 case of the same recipe (100,352 elements, 210.40 MB read +
    # 2.19 MB written per launch, two launches) and scaled to 131,072 elements; both
    # kernels below are unchanged since their captures (the hash is of the file, in
    # which other kernels changed)
    "plain": {"kernel": "jacobi_kernel<float,10,0>", "file": "kernels_mv.cu",
              "src_sha": "e49eeb68f4ccb194",
              "bytes_per_launch": (210.40e6 + 2.19e6) * 131072 / 100352},
    "tma": {"kernel": "jacobi_tma_kernel<float,10>", "file": "kernels_tma.cu",
            "src_sha": "24cbc7a902631ea2", "bytes_per_launch": 274.87e6 + 6.52e6},
    # folded step x + c - (wD^-1 A) x, two blocks of a row in flight: captured at full
    # size on the benchmark's block pattern (csrc/bench_level0.cu, 131,072 block rows;
    # 222.42 MB read + 3.81 MB written per launch)
    "folded": {"kernel": "folded_pair_kernel<10,6>", "file": "kernels_mv.cu",
               "src_sha": "e49eeb68f4ccb194",
               "bytes_per_launch": 222.42e6 + 3.81e6},
}


def src_hash(name):
    with open(os.path.join(ROOT, "paper_2504_13373_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per side (default: the full workload)")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-iters", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-warmup", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="one mixed solve only (for an ncu launch list); prints no bench line")
    ap.add_argument("--host-loop", action="store_true",
                    help="with --profile-run: drive the CG loop from the host (per-kernel ncu)")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="with --profile-run: stop each solve after this many CG iterations")
    ap.add_argument("--folded-smoother", type=int, default=-1, choices=[-1, 0, 1],
                    help="level-0 steps as x + c - (wD^-1 A) x (1) or x + wD^-1 (b - A x) (0); "
                         "-1: the library default")
    ap.add_argument("--dense-tail-dofs", type=int, default=-1,
                    help="coarse levels of at most this many dofs as one dense operator "
                         "(0: off); -1: the library default")
    ap.add_argument("--fused-restriction", type=int, default=-1, choices=[-1, 0, 1],
                    help="residual and restriction fused through R A (1) or as two steps (0); "
                         "-1: the library default")
    ap.add_argument("--grid-tail", type=int, default=-1, choices=[-1, 0, 1],
                    help="coarse levels as one persistent launch (1) or one launch per step (0); "
                         "-1: the library default")
    ap.add_argument("--bulk-staging", action="store_true",
                    help="level-0 FP32 sweep with bulk-copy (TMA) staging of A and w D^-1")
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="requests of the serving stream (0: skip the serving measurement)")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4"],
                    help="c2 (default): the P3 256^2 bench line; c1 / c3 / c4: solves/s of the "
                         "P1 32^2, LDG Q2 512^2 conv-diff and P2 48^3 tet workloads per precision")
    ap.add_argument("--peclet", type=float, default=100.0, help="Peclet number of c3")
    ap.add_argument("--matrix-free-levels", type=int, default=0,
                    help="with --workload: levels 1..k applied matrix-free (Section 4.4)")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the c1 / c3 / c4 records of the default run")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(v, dist, device=None):
    """The slowest rank's time (every rank gets it); `dist` is
    torch.distributed or None for one process."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_problem(n):
    from synth import configs
    return configs.poisson2d_p3(n=n)


def hbm_peak():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------
# algorithmic bytes of one preconditioned CG iteration (whole-iteration roofline)
# ----------------------------------------------------------------------------
def level_shapes(gasa, ctx, n_levels):
    """gasa_level_shape per level, plus RA_nnzb: the blocks of R_k A_k where the
    fused restriction keeps it (0 elsewhere), and dense_tail: True on the first
    level of the dense bottom operator (levels k .. N as one dense product)."""
    cyc = gasa.gasa_cycle_info(ctx)
    shapes = []
    for k in range(n_levels):
        sh = dict(gasa.gasa_level_shape(ctx, k))
        sh["RA_nnzb"] = 0
        if k < n_levels - 1:
            n_next = gasa.gasa_level_shape(ctx, k + 1)["units"]
            try:
                rp = gasa.gasa_get_level(ctx, k, gasa.GASA_LV_RA_ROWPTR, np.zeros(n_next + 1, np.int32))
                sh["RA_nnzb"] = int(rp[-1])
            except gasa.GasaError:
                pass
        sh["dense_tail"] = cyc["dense_n"] > 0 and k == cyc["dense_first_level"]
        sh["folded"] = k == 0 and cyc["folded"] == 1
        shapes.append(sh)
    return shapes


def _fused_first(s_next, s, n_next, nnzb, w):
    """whether the FP32 fused restriction also takes the next level's first
    smoothing step: the lane-team kernel (square blocks of 2..8 with >= 6
    blocks of R and R A per row) or the wide-block kernel (> 8 rows or
    columns, at most 40, >= 8 per row)"""
    if w != 4:
        return False
    if s_next == s and 2 <= s <= 8 and nnzb >= 6 * n_next:
        return True
    return (s_next > 8 or s > 8) and s_next <= 40 and s <= 40 and nnzb >= 8 * n_next


def iteration_bytes(shapes, precision, t_pre=3, t_post=3):
    """Bytes one CG iteration must move, counted once per kernel that reads
    or writes them (matrix values, column indices and row pointers, the
    vectors each kernel touches), for the kernels a graph-resident CG step
    launches: the V-cycle of Alg. 2 on every level (first pre-smoothing step
    x = w D^-1 b, t_pre - 1 further sweeps, residual, restriction, coarsest
    dense solve, prolongation, t_post sweeps), the outer product q = A p and
    the CG vector updates with their dot products.  precision: 'fp64',
    'mixed32' (FP32 V-cycle, double-single outer product) or 'mixed16'
    (as mixed32 with FP16 level-0 A and w D^-1 plus one FP32 scale per
    block).  Where the hierarchy has a dense bottom from level kt, levels
    kt .. N cost one dense FP64 product (n_kt^2 * 8 bytes and the two
    vectors); with the folded level-0 smoother its later steps read W A and c
    in place of A, W and b.  Returns (total bytes, per-part dict)."""
    N = len(shapes) - 1
    w = 8 if precision == "fp64" else 4
    parts = {}
    n0 = shapes[0]["units"] * shapes[0]["s"]
    first_done = [False] * (N + 1)
    kt = next((k for k in range(N + 1) if shapes[k].get("dense_tail")), N)
    for k in range(kt):
        sh = shapes[k]
        n, s, nnzb = sh["units"], sh["s"], sh["nnzb"]
        nxt = shapes[k + 1]
        n1, s1 = nxt["units"], nxt["s"]
        wa = 2 if (precision == "mixed16" and k == 0) else w
        scale = 4 if (precision == "mixed16" and k == 0) else 0
        A = nnzb * (s * s * wa + scale) + 4 * nnzb + 4 * (n + 1)
        W = n * (s * s * wa + scale)
        v = n * s * w
        R = sh["R_nnzb"] * (s * s1 * w) + 4 * sh["R_nnzb"] + 4 * (n1 + 1)
        P = sh["P_nnzb"] * (s * s1 * w) + 4 * sh["P_nnzb"] + 4 * (n + 1)
        folded = bool(sh.get("folded")) and precision == "mixed32"
        first = W + 2 * v
        if k == 0 and precision == "mixed32":
            first = W + n * s * (8 + 4 + 4)      # reads the FP64 residual, writes x and its FP32 copy
        if folded:
            first += v                            # also keeps c = W b
        if first_done[k]:
            first = 0.0                           # taken by the restriction of the level above
        # folded steps u + c - (W A) u read W A (A's size) and c, not A, W and b
        sweeps = (t_pre - 1 + t_post) * ((A if folded else A + W) + 3 * v)
        ra = sh.get("RA_nnzb", 0)
        if ra and not (precision == "mixed16" and k == 0):
            # fused: b_{k+1} = R b - (R A) x, maybe with level k+1's first step
            RAb = ra * (s1 * s * w) + 4 * ra + 4 * (n1 + 1)
            resid = 0.0
            restrict = R + RAb + 2 * v + n1 * s1 * w
            if k + 1 < kt and _fused_first(s1, s, n1, sh["R_nnzb"] + ra, w):
                restrict += n1 * s1 * s1 * w + n1 * s1 * w
                first_done[k + 1] = True
        else:
            resid = A + 3 * v
            restrict = R + v + n1 * s1 * w
        prolong = P + n1 * s1 * w + 2 * v
        parts[f"level{k}"] = first + sweeps + resid + restrict + prolong
    nc = shapes[kt]["units"] * shapes[kt]["s"]
    parts["coarse" if kt == N else "dense_tail"] = nc * nc * 8 + 2 * nc * w
    sh = shapes[0]
    nnzb, s, n = sh["nnzb"], sh["s"], sh["units"]
    idx = 4 * nnzb + 4 * (n + 1)
    if precision == "fp64":
        parts["outer_Ap"] = nnzb * s * s * 8 + idx + 2 * n0 * 8
        parts["vectors"] = 2 * n0 * 8 + 2 * 2 * n0 * 8 + 3 * n0 * 8 + 6 * n0 * 8
        # p.q dot; r.z dot; p = z + beta p (2 reads, 1 write); x, r update (4 reads, 2 writes)
    else:
        parts["outer_Ap"] = nnzb * s * s * 8 + idx + n0 * (8 + 8 + 8)
        # A hi + lo words; p hi + lo gathered once, q written, p read for p.q
        parts["vectors"] = (n0 * (8 + 4 + 4)                # r.z and r.zold in one pass (z, zold FP32)
                            + n0 * (4 + 8 + 8 + 4 + 4 + 4)    # p = z + beta p, zold = z, p's hi/lo split
                            + 6 * n0 * 8)                     # x, r update
    return float(sum(parts.values())), {k: float(v) for k, v in parts.items()}


def gmres_iteration_bytes(shapes, precision, iterations, restart=30, t_pre=3, t_post=3):
    """Average bytes of one GMRES(restart) step (flexible for the mixed
    V-cycles) over a solve of `iterations` steps: the V-cycle (with the FP64 /
    FP32 conversions around an FP32 one), the FP64 outer product, classical
    Gram-Schmidt applied twice against the j + 1 basis vectors of step j
    (a multi-dot reading the basis and w, an update reading the basis and w
    and writing w, per pass), the norm and the normalisation into v_{j+1}.
    Restart overheads (a residual, a norm and the combination of the basis)
    are spread over the steps of their cycle."""
    tot, parts = iteration_bytes(shapes, "fp64" if precision == "fp64" else precision, t_pre, t_post)
    vc = sum(v for k, v in parts.items() if k.startswith("level") or k in ("coarse", "dense_tail"))
    sh = shapes[0]
    nnzb, s, n = sh["nnzb"], sh["s"], sh["units"]
    n0 = n * s
    spmv = nnzb * s * s * 8 + 4 * nnzb + 4 * (n + 1) + 2 * n0 * 8
    conv = 0 if precision == "fp64" else n0 * (8 + 4) + n0 * (4 + 8)
    steps, js = 0, []
    while steps < iterations:
        m = min(restart, iterations - steps)
        js.append(list(range(m)))
        steps += m
    total = 0.0
    for cyc in js:
        for j in cyc:
            arnoldi = 2 * ((j + 2) + (j + 3)) * n0 * 8 + 3 * n0 * 8
            total += vc + conv + spmv + arnoldi
        m = len(cyc)
        total += (spmv + n0 * 8) + (m + 2) * n0 * 8        # restart residual + norm, combine
    return total / max(1, iterations)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region; the SM clock
    reported is the median over the samples taken under load (GPU utilisation
    of at least 50 %), throttle reasons are collected over every sample."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")
    LOAD_UTIL = 50.0

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = tempfile.mktemp(prefix="gasa_clk_", suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        with open(self.path) as f:
            out = self.parse(f)
        os.unlink(self.path)
        return out

    @classmethod
    def parse(cls, lines):
        sm, mx, loaded, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 7:
                continue
            try:
                clk, clk_max = float(p[0]), float(p[1])
            except ValueError:
                continue
            sm.append(clk)
            mx.append(clk_max)
            try:
                if len(p) > 7 and float(p[7]) >= cls.LOAD_UTIL:
                    loaded.append(clk)
            except ValueError:
                pass
            for nm, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(loaded if loaded else sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm), "samples_under_load": len(loaded)}


# ----------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline leg and --impl reference)
# ----------------------------------------------------------------------------
ORACLE_SOLVE = os.path.join(ROOT, "tests", "golden", "c2_oracle_solve.json")


def oracle_solve_record():
    """The oracle's own solves of the full workload (iterations, residuals,
    sampled x), written by tests/golden/make_c2_oracle_solve.py; None when
    absent."""
    try:
        with open(ORACLE_SOLVE) as f:
            return json.load(f)
    except Exception:
        return None


def cpu_sample_main(path, warmup, iters):
    """Runs in a single-threaded child: oracle setup on the saved workload
    (untimed), `warmup` untimed flexible-CG iterations with the float32
    V-cycle, then `iters` timed ones (one timer per iteration)."""
    from oracle import gasa_oracle as O
    d = np.load(path, allow_pickle=True)
    aggs = [d[f"agg{k}"] for k in range(int(d["nagg"]))]
    t0 = time.perf_counter()
    H = O.setup(d["row_ptr"], d["col"], d["val"], aggs, B0=d["B0"], r=int(d["r"]), dim=2)
    t_setup = time.perf_counter() - t0
    M = O.make_vcycle(H, "fp32")
    A = H.levels[0].A
    if warmup > 0:
        O.pcg(A, d["rhs"], M, 1e-300, warmup, flexible=True)
    t0 = time.perf_counter()
    O.pcg(A, d["rhs"], M, 1e-300, iters, flexible=True)
    total = time.perf_counter() - t0
    print(json.dumps({"setup_s": t_setup, "s_per_iter": total / iters, "timed_s": total,
                      "iters": iters}))


def run_cpu_sample(pr, iters, warmup=0):
    tmp = tempfile.mktemp(prefix="gasa_wl_", suffix=".npz")
    np.savez(tmp, row_ptr=pr.A.row_ptr, col=pr.A.col, val=pr.A.val, B0=pr.B0, r=pr.r,
             rhs=pr.rhs, nagg=len(pr.agg_of), **{f"agg{k}": a for k, a in enumerate(pr.agg_of)})
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", tmp,
                              "--cpu-iters", str(iters), "--cpu-warmup", str(warmup)],
                             capture_output=True, text=True, env=env, timeout=1800)
        line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
        if out.returncode != 0 or not line:
            return None, out.stderr[-2000:]
        return json.loads(line[-1]), None
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)


# ----------------------------------------------------------------------------
def main():
    args = parse()
    if args.cpu_sample:
        cpu_sample_main(args.cpu_sample, args.cpu_warmup, args.cpu_iters)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_main(args, rank, world)
    if args.workload != "c2":
        return workload_main(args, local) if rank == 0 else 0
    return ours_main(args, rank, world, local)


def reference_main(args, rank, world):
    """The reference arm is the CPU oracle as it stands, on one host core.
    One step is one flexible-CG iteration of the oracle (float32 V-cycle) on
    the full workload, timed; W untimed iterations come first.  A whole
    solve takes the oracle's own iteration count, from its committed run to
    1e-10 (tests/golden/c2_oracle_solve.json), so solves/s = 1 / (seconds per
    iteration x that count).  Under torchrun only rank 0 runs."""
    if rank != 0:
        return 0
    pr = build_problem(args.n)
    rec = oracle_solve_record()
    iters_per_solve = None
    if rec is not None and rec.get("dofs") == pr.n_dofs and "mixed32" in rec:
        iters_per_solve = int(rec["mixed32"]["iterations"])
    steps = max(1, args.steps)
    res, err = run_cpu_sample(pr, steps, max(0, args.warmup))
    if res is None or iters_per_solve is None:
        why = f"oracle sample failed: {err}" if res is None else \
            "no committed oracle solve of this workload (tests/golden/c2_oracle_solve.json)"
        print(json.dumps({"impl": "reference", "unavailable": why}))
        return 0
    value = 1.0 / (res["s_per_iter"] * iters_per_solve)
    sample = (f"oracle setup on the full workload ({res['setup_s']:.1f} s, untimed), "
              f"{max(0, args.warmup)} untimed and {steps} timed flexible-CG iterations with the "
              f"float32 V-cycle ({res['s_per_iter']:.3f} s each); a solve = {iters_per_solve} "
              f"iterations, the oracle's own count to 1e-10 from its committed full run")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": res["s_per_iter"] * 1e3,
        "step": "one flexible-CG iteration of the oracle (float32 V-cycle) on the full workload",
        "iterations_per_solve": iters_per_solve,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": args.n},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))
    return 0


def serve_bench(gasa, n_requests, device=0):
    """Serving stream: 8 resident meshes (2D/3D SIPG Poisson and 2D LDG
    convection-diffusion, P1-P3, 1e3-2e6 dofs), requests with N(0,1)
    right-hand sides.  Saturated throughput with every request queued at
    once, then open-loop Poisson arrivals at 0.5x and 1.5x that rate; latency
    is submit-to-completion as the server records it."""
    from synth import configs, serving
    seed = configs.SEED
    t0 = time.perf_counter()
    specs = serving.mesh_specs(seed)
    probs = [serving.build_mesh(sp, seed) for sp in specs]
    t_gen = time.perf_counter() - t0
    ctxs, setup_s, hier_bytes = [], [], []
    for pr in probs:
        ctx = gasa.gasa_create(device)
        opt = gasa.gasa_default_options(dim=pr.dim, n_cand=pr.r, max_iter=20000,
                                        solver=gasa.GASA_SOLVER_CG if pr.solver == "cg"
                                        else gasa.GASA_SOLVER_GMRES)
        info = gasa.gasa_setup(ctx, pr.A.row_ptr, pr.A.col, pr.A.val.ravel(), pr.A.b, pr.agg_of,
                               opt, adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx,
                               centroids=pr.centroids, init_candidates=pr.B0)
        ctxs.append(ctx)
        setup_s.append(info.seconds)
        hier_bytes.append(info.device_bytes)
    which = serving.request_mesh(seed, n_requests)
    rhs = [serving.request_rhs(seed, i, probs[m].n_dofs) for i, m in enumerate(which)]
    budget = 40 << 30
    srv = gasa.gasa_server_create(device, budget, 8)
    out = {"meshes": [dict(name=sp.name, dofs=sp.dofs, levels=pr.n_levels, r=pr.r,
                           solver=pr.solver, setup_s=su)
                      for sp, pr, su in zip(specs, probs, setup_s)],
           "requests": n_requests, "budget_bytes": budget, "max_batch": 8,
           "generate_s": t_gen}
    try:
        ids = [gasa.gasa_server_add_mesh(srv, c) for c in ctxs]

        def run(prec, times=None):
            """Submit every request (at `times` seconds from the start if
            given), wait for all; (wall seconds, latencies, iterations)."""
            tickets = []
            start = time.perf_counter()
            for i, m in enumerate(which):
                if times is not None:
                    wait = start + times[i] - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                tickets.append(gasa.gasa_server_submit(srv, ids[m], rhs[i], TOL, prec))
            gasa.gasa_server_drain(srv, 1800.0)
            wall = time.perf_counter() - start
            lat, its, worst = [], [], 0.0
            for t in tickets:
                st, info = gasa.gasa_server_poll(srv, t)
                if st != gasa.GASA_OK:
                    raise RuntimeError(f"served solve failed: {gasa.gasa_status_string(st)}")
                lat.append(info.seconds * 1e3)
                its.append(info.iterations)
                worst = max(worst, info.rel_residual)
            return wall, np.array(lat), np.array(its), worst

        for name, prec in (("mixed", gasa.GASA_PREC_MIXED32), ("fp64", gasa.GASA_PREC_FP64)):
            # warm-up: one request per mesh creates the engines and their graphs
            for m in range(len(ctxs)):
                gasa.gasa_server_submit(srv, ids[m], serving.request_rhs(seed, 10 ** 6 + m,
                                                                         probs[m].n_dofs), TOL, prec)
            gasa.gasa_server_drain(srv, 600.0)
            st0 = gasa.gasa_server_stats_read(srv)
            wall, lat, its, worst = run(prec)
            sat = n_requests / wall
            res = {"saturated": {"solves_per_s": sat, "wall_s": wall,
                                 "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99))},
                   "iterations_median": float(np.median(its)), "rel_residual_max": worst,
                   "per_mesh": {specs[m].name: {"requests": int((which == m).sum()),
                                                "iterations_median": float(np.median(its[which == m])),
                                                "iterations_max": int(its[which == m].max()),
                                                "latency_p50_ms": float(np.percentile(lat[which == m], 50))}
                                for m in range(len(specs)) if (which == m).any()}}
            for f in (0.5, 1.5):
                times = serving.arrival_times(seed, n_requests, f * sat)
                wall, lat, its, worst = run(prec, times)
                small = np.array([specs[m].dofs < 20000 for m in which])
                res[f"open_loop_{f:g}x"] = {
                    "rate_per_s": f * sat, "solves_per_s": n_requests / wall,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "p50_ms_meshes_under_2e4_dofs": (float(np.percentile(lat[small], 50))
                                                     if small.any() else None),
                    "per_mesh_p50_ms": {specs[m].name: float(np.percentile(lat[which == m], 50))
                                        for m in range(len(specs)) if (which == m).any()}}
                res["rel_residual_max"] = max(res["rel_residual_max"], worst)
            st1 = gasa.gasa_server_stats_read(srv)
            res["graph_launches"] = st1["graph_launches"] - st0["graph_launches"]
            res["peak_running"] = st1["peak_running"]
            out[name] = res
        out["peak_bytes"] = gasa.gasa_server_stats_read(srv)["peak_bytes"]
    finally:
        gasa.gasa_server_destroy(srv)
        for c in ctxs:
            gasa.gasa_destroy(c)
    return out


def build_workload(which, n_arg=None, peclet=100.0):
    from synth import configs
    if which == "c1":
        return configs.poisson2d_p1(), "poisson2d_sipg_p1_tri_32x32"
    if which == "c3":
        n = n_arg or 512
        return (configs.convdiff2d_q2(n=n, peclet=peclet),
                f"convdiff2d_ldg_q2_quad_{n}x{n}_pe{peclet:g}")
    n = n_arg or 48
    return configs.poisson3d_p2(n=n), f"poisson3d_sipg_p2_tet_{n}cubed"


def measure_workload(gasa, pr, name, steps, warmup, device, opt_kw=None):
    """solves/s, iterations, true residual, error against this run's FP64
    solve and a whole-iteration roofline of one workload, per precision:
    FP64, FP32 V-cycle, FP16-block V-cycle (the parity tests pin each
    precision's solve to the oracle's on reduced sizes of the same recipe).
    opt_kw: further gasa_options fields (the roofline's byte model counts
    stored operators, so it overstates matrix-free levels' bytes)."""
    import torch
    A = pr.A
    ctx = gasa.gasa_create(device)
    opt = gasa.gasa_default_options(dim=pr.dim, n_cand=pr.r, max_iter=20000,
                                    solver=gasa.GASA_SOLVER_CG if pr.solver == "cg"
                                    else gasa.GASA_SOLVER_GMRES, **(opt_kw or {}))
    sinfo = gasa.gasa_setup(ctx, A.row_ptr, A.col, A.val.ravel(), A.b, pr.agg_of, opt,
                            adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx, centroids=pr.centroids,
                            init_candidates=pr.B0)
    shapes = level_shapes(gasa, ctx, sinfo.n_levels)
    dense_tail = gasa.gasa_cycle_info(ctx)
    peak, peak_kind = hbm_peak()
    b = torch.from_numpy(pr.rhs).cuda(device)
    x = torch.zeros_like(b)
    out, x64 = {}, None
    As = A.to_scipy()
    try:
        for pname, prec in (("fp64", gasa.GASA_PREC_FP64), ("mixed32", gasa.GASA_PREC_MIXED32),
                            ("mixed16", gasa.GASA_PREC_MIXED16)):
            for _ in range(warmup):
                gasa.gasa_solve(ctx, b, x, TOL, prec, on_device=True)
            torch.cuda.synchronize()
            per, infos = [], []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                infos.append(gasa.gasa_solve(ctx, b, x, TOL, prec, on_device=True))
                e1.record()
                torch.cuda.synchronize()
                per.append(e0.elapsed_time(e1))
            xh = x.cpu().numpy()
            if x64 is None:
                x64 = xh.copy()
            its = int(infos[-1].iterations)
            ms = float(np.median(per))
            if pr.solver == "cg":
                b_it = iteration_bytes(shapes, pname, opt.t_pre, opt.t_post)[0]
            else:
                b_it = gmres_iteration_bytes(shapes, pname, its, opt.restart or 30, opt.t_pre, opt.t_post)
            gbs = b_it / (ms / max(1, its) / 1e3) / 1e9
            out[pname] = {
                "solves_per_s": 1e3 / ms, "median_ms": ms, "iterations": its,
                "rel_residual": float(np.linalg.norm(pr.rhs - As @ xh) / np.linalg.norm(pr.rhs)),
                "rel_err_vs_fp64_solve": float(np.linalg.norm(xh - x64) / np.linalg.norm(x64)),
                "roofline_iteration": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                       "frac": gbs / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                                       "bytes_per_iteration": b_it,
                                       "ms_per_iteration": ms / max(1, its)}}
    finally:
        gasa.gasa_destroy(ctx)
    return {"workload": name, "dofs": pr.n_dofs, "block": A.b, "nnzb": int(A.nnzb),
            "levels": sinfo.n_levels, "candidates": pr.r, "solver": pr.solver,
            "level_dofs": [int(sinfo.dofs[k]) for k in range(sinfo.n_levels)],
            "level_nnzb": [int(sinfo.nnzb[k]) for k in range(sinfo.n_levels)],
            "level_block": [int(sinfo.block[k]) for k in range(sinfo.n_levels)],
            "cycle": dense_tail, "options": dict(opt_kw or {}),
            "device_bytes": int(sinfo.device_bytes), "setup_s": sinfo.seconds, "steps": steps, "warmup": warmup, "precisions": out}


def other_workloads(gasa, device, steps=1, warmup=1):
    """The P1 32^2 workload, the LDG + upwind Q2 512^2 workload at Peclet 1,
    100 and 1e4, and the P2 48^3 tet workload, one record each."""
    recs = []
    for which, pe in (("c1", None), ("c3", 1.0), ("c3", 100.0), ("c3", 1e4), ("c4", None)):
        t0 = time.perf_counter()
        pr, name = build_workload(which, None, pe if pe is not None else 100.0)
        t_gen = time.perf_counter() - t0
        rec = measure_workload(gasa, pr, name, steps, warmup, device)
        rec["generate_s"] = t_gen
        recs.append(rec)
        del pr
    return recs


def workload_main(args, local):
    """--workload c1 / c3 / c4: one workload's record, as a bench line."""
    import torch
    from paper_2504_13373_gb300 import gasa
    gasa.load()
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    n_arg = None if args.n == 256 else args.n
    pr, name = build_workload(args.workload, n_arg, args.peclet)
    t_gen = time.perf_counter() - t0
    if args.profile_run:
        # one mixed solve from the host-driven loop (per-kernel ncu launch list)
        A = pr.A
        ctx = gasa.gasa_create(local)
        opt = gasa.gasa_default_options(dim=pr.dim, n_cand=pr.r, max_iter=20000,
                                        solver=gasa.GASA_SOLVER_CG if pr.solver == "cg"
                                        else gasa.GASA_SOLVER_GMRES)
        if args.profile_iters > 0:
            opt.max_iter = args.profile_iters
        gasa.gasa_setup(ctx, A.row_ptr, A.col, A.val.ravel(), A.b, pr.agg_of, opt,
                        adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx, centroids=pr.centroids,
                        init_candidates=pr.B0)
        b = torch.from_numpy(pr.rhs).cuda()
        x = torch.zeros_like(b)
        # launches before the solve, for an ncu skip count (-s)
        print(json.dumps({"setup_launches": gasa.gasa_kernel_launches()}), flush=True)
        gasa.gasa_profile_enable(ctx, True)
        gasa.gasa_solve(ctx, b, x, TOL, gasa.GASA_PREC_MIXED32, on_device=True,
                        allow_not_converged=args.profile_iters > 0)
        torch.cuda.synchronize()
        gasa.gasa_destroy(ctx)
        return 0
    with ClockSampler(local) as clk:
        kw = {"matrix_free_levels": args.matrix_free_levels} if args.matrix_free_levels > 0 else None
        rec = measure_workload(gasa, pr, name, args.steps, args.warmup, local, kw)
    mix = rec["precisions"]["mixed32"]
    print(json.dumps({
        "metric": METRIC, "value": mix["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mix["median_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": {"workload": name, "tol": TOL},
        "record": rec, "generate_s": t_gen, "clocks": clk.summary()}))
    return 0


def ours_main(args, rank, world, local):
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2504_13373_gb300 import gasa
    gasa.load()

    t0 = time.perf_counter()
    pr = build_problem(args.n)
    t_gen = time.perf_counter() - t0
    A = pr.A
    n = pr.n_dofs
    stream = torch.cuda.Stream()
    ctx = gasa.gasa_create(local, stream)
    opt = gasa.gasa_default_options(dim=2, n_cand=pr.r, max_iter=20000)
    if args.profile_run and args.profile_iters > 0:
        opt.max_iter = args.profile_iters
    if args.grid_tail >= 0:
        opt.grid_tail = args.grid_tail
    if args.fused_restriction >= 0:
        opt.fused_restriction = args.fused_restriction
    if args.dense_tail_dofs >= 0:
        opt.dense_tail_dofs = args.dense_tail_dofs
    if args.folded_smoother >= 0:
        opt.folded_smoother = args.folded_smoother
    opt.bulk_staging = 1 if args.bulk_staging else 0
    sinfo = gasa.gasa_setup(ctx, A.row_ptr, A.col, A.val.ravel(), A.b, pr.agg_of, opt,
                            adj_ptr=pr.adj_ptr, adj_idx=pr.adj_idx, centroids=pr.centroids,
                            init_candidates=pr.B0)
    b_dev = torch.from_numpy(pr.rhs).to(f"cuda:{local}")
    x_dev = torch.zeros_like(b_dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(precision, steps, profile=False):
        """K solves bracketed by events on the library's stream."""
        infos = []
        per = []
        barrier()
        if profile:
            gasa.gasa_profile_enable(ctx, True)
        l0 = gasa.gasa_kernel_launches()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(steps):
                e_a = torch.cuda.Event(enable_timing=True)
                e_b = torch.cuda.Event(enable_timing=True)
                e_a.record(stream)
                infos.append(gasa.gasa_solve(ctx, b_dev, x_dev, TOL, precision, on_device=True))
                e_b.record(stream)
                per.append((e_a, e_b))
            ev1.record(stream)
        stream.synchronize()
        launches = gasa.gasa_kernel_launches() - l0
        ms = ev0.elapsed_time(ev1)
        per_ms = [a.elapsed_time(bb) for a, bb in per]
        barrier()
        ms = max_over_ranks(ms, dist, f"cuda:{local}")
        return ms, infos, launches, per_ms

    if args.profile_run:
        # launches before the first solve, for an ncu skip count (-s)
        print(json.dumps({"setup_launches": gasa.gasa_kernel_launches()}), flush=True)
        if args.host_loop:
            # kernel nodes inside a graph with conditional nodes cannot be
            # profiled one by one; the host-driven loop runs the same kernels
            gasa.gasa_profile_enable(ctx, True)
        for _ in range(max(1, args.steps)):
            gasa.gasa_solve(ctx, b_dev, x_dev, TOL, gasa.GASA_PREC_MIXED32, on_device=True,
                            allow_not_converged=args.profile_iters > 0)
        torch.cuda.synchronize()
        gasa.gasa_destroy(ctx)
        return 0
    # warm-up
    for _ in range(args.warmup):
        gasa.gasa_solve(ctx, b_dev, x_dev, TOL, gasa.GASA_PREC_MIXED32, on_device=True)
        gasa.gasa_solve(ctx, b_dev, x_dev, TOL, gasa.GASA_PREC_FP64, on_device=True)
    xs = {}
    with ClockSampler(local) as clk:
        ms_mix, inf_mix, launches, per_mix = timed(gasa.GASA_PREC_MIXED32, args.steps)
        xs["mixed32"] = x_dev.cpu().numpy()
        ms_64, inf_64, _, per_64 = timed(gasa.GASA_PREC_FP64, args.steps)
        xs["fp64"] = x_dev.cpu().numpy()
        ms_16, inf_16, _, per_16 = timed(gasa.GASA_PREC_MIXED16, args.steps)
        xs["mixed16"] = x_dev.cpu().numpy()
        # roofline of the dominant kernel: one more mixed solve with CUDA events
        # around every level-0 sweep (events cannot sit inside the solve graph,
        # so this solve runs the same kernels from the host-driven loop)
        _, inf_prof, _, _ = timed(gasa.GASA_PREC_MIXED32, 1, profile=True)
        prof = gasa.gasa_profile_read(ctx, 0)
        prof_all = {name: gasa.gasa_profile_read(ctx, c) for c, name in enumerate(PROFILE_CLASSES)}
        gasa.gasa_profile_enable(ctx, False)
    clocks = clk.summary()
    # true residual of the last solves, checked on the host
    x_host = x_dev.cpu().numpy()
    # end to end through the public call with host buffers (pinned)
    b_pin = torch.from_numpy(pr.rhs).pin_memory()
    x_pin = torch.zeros(n, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        inf_e2e = gasa.gasa_solve(ctx, b_pin, x_pin, TOL, gasa.GASA_PREC_MIXED32, on_device=False)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, f"cuda:{local}")
    rel_host = float(np.linalg.norm(pr.rhs - A.to_scipy() @ x_pin.numpy()) / np.linalg.norm(pr.rhs))

    value = world * args.steps / (ms_mix / 1e3)
    value64 = world * args.steps / (ms_64 / 1e3)
    ms_k, n_k, bytes_k = prof
    achieved = (bytes_k / n_k) / (ms_k / n_k / 1e3) / 1e9 if n_k else None
    iters = [i.iterations for i in inf_mix]
    shapes = level_shapes(gasa, ctx, sinfo.n_levels)
    sweep_form = "tma" if args.bulk_staging else ("folded" if shapes[0]["folded"] else "plain")
    ncu = NCU_TRAFFIC[sweep_form]
    traffic = ncu["bytes_per_launch"] if ncu["src_sha"] == src_hash(ncu["file"]) else None

    def iteration_roofline(prec, ms, infos):
        """algorithmic bytes of one CG iteration / (solve time / iterations)"""
        b_it, parts = iteration_bytes(shapes, prec, opt.t_pre, opt.t_post)
        ms_it = ms / max(1, sum(i.iterations for i in infos))
        gbs = b_it / (ms_it / 1e3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "peak_kind": f"{peak_kind} hbm_gbs", "bytes_per_iteration": b_it,
                "ms_per_iteration": ms_it, "bytes_by_part": parts,
                "what": "whole preconditioned CG iteration (V-cycle on every level, outer A p, "
                        "vector updates and dot products); time = timed solves / their iterations"}

    peak, peak_kind = hbm_peak()
    roof_it = {"mixed32": iteration_roofline("mixed32", ms_mix, inf_mix),
               "fp64": iteration_roofline("fp64", ms_64, inf_64),
               "mixed16": iteration_roofline("mixed16", ms_16, inf_16)}
    err_vs_oracle = None
    rec0 = oracle_solve_record()
    if rec0 is not None and rec0.get("dofs") == n and "fp64" in rec0:
        idx = np.asarray(rec0["sample_index"], dtype=np.int64)
        xo = np.asarray(rec0["fp64"]["x_sample"])
        err_vs_oracle = {
            "what": ("||x - x_oracle|| / ||x_oracle|| over the 4,096 sampled dofs of the oracle's "
                     "own FP64 solve (tests/golden/c2_oracle_solve.json)"),
            **{k: float(np.linalg.norm(v[idx] - xo) / np.linalg.norm(xo)) for k, v in xs.items()}}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_mix / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD if args.n == 256 else f"poisson2d_sipg_p3_tri_{args.n}x{args.n}",
            "dofs": n, "elements": A.n, "block": A.b, "nnzb": int(A.nnzb), "levels": sinfo.n_levels,
            "candidates": pr.r, "tol": TOL, "solver": "CG (flexible for mixed)",
            "cycle": gasa.gasa_cycle_info(ctx),
            "l2": "inputs larger than L2 (A 419 MB FP64 / 209 MB FP32 per pass), no flush",
            "parallelism": f"replicas x{world}",
        },
        "iterations": {"mixed": iters, "fp64": [i.iterations for i in inf_64]},
        "rel_residual": {"mixed": max(i.rel_residual for i in inf_mix),
                         "fp64": max(i.rel_residual for i in inf_64), "e2e_host_check": rel_host},
        "fp64": {"value": value64, "unit": "solves/s", "ms_per_step": ms_64 / args.steps,
                 "p50_ms": float(np.percentile(per_64, 50)), "p99_ms": float(np.percentile(per_64, 99))},
        "mixed16": {"value": world * args.steps / (ms_16 / 1e3), "unit": "solves/s",
                    "ms_per_step": ms_16 / args.steps, "iterations": [i.iterations for i in inf_16],
                    "rel_residual": max(i.rel_residual for i in inf_16),
                    "storage": "level-0 A and wD^-1 as FP16 blocks with one FP32 scale per block"},
        "p50_ms": float(np.percentile(per_mix, 50)),
        "p99_ms": float(np.percentile(per_mix, 99)),
        "setup_s": sinfo.seconds,
        "generate_s": t_gen,
        "roofline": {"kernel": (f"level-0 block-Jacobi step x + c - (wD^-1 A) x, c = wD^-1 b, FP32 ({ncu['kernel']})"
                                if sweep_form == "folded" else
                                f"level-0 block-Jacobi step x + wD^-1(b - Ax), FP32 ({ncu['kernel']})"),
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_k / n_k if n_k else None,
                     "launches": n_k, "avg_launch_us": ms_k / n_k * 1e3 if n_k else None},
        "roofline_iteration": roof_it,
        "level0_kernels": {
            name: {"avg_us": ms / n * 1e3, "launches": n, "algorithmic_bytes_per_launch": by / n,
                   "achieved_gbs": by / n / (ms / n / 1e3) / 1e9,
                   "frac": by / n / (ms / n / 1e3) / 1e9 / peak}
            for name, (ms, n, by) in prof_all.items() if n},
        "error_vs_oracle": err_vs_oracle,
        "e2e": {"value": world * args.steps / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    rec = oracle_solve_record()
    oracle_iters = None
    if rec is not None and rec.get("dofs") == n and "mixed32" in rec:
        oracle_iters = int(rec["mixed32"]["iterations"])
        line["oracle"] = {k: {"iterations": rec[k]["iterations"], "rel_residual": rec[k]["rel_residual"]}
                          for k in ("fp64", "mixed32", "mixed16") if k in rec}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res, err = run_cpu_sample(pr, args.cpu_iters)
        per_solve = oracle_iters or int(np.median(iters))
        if res is not None:
            sps = 1.0 / (res["s_per_iter"] * per_solve)
            line["cpu_baseline"] = {
                "value": sps, "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": (f"oracle setup on the full workload ({res['setup_s']:.1f} s, untimed), then "
                           f"{args.cpu_iters} flexible-CG iterations with the float32 V-cycle at "
                           f"{res['s_per_iter']:.3f} s each, scaled to {per_solve} iterations per "
                           f"solve (" + ("the oracle's own count from its committed full run"
                                         if oracle_iters else "this run's count") + ")")}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {err}"}
    gasa.gasa_destroy(ctx)
    if args.serve_requests > 0 and world == 1:
        # the serving stream is a per-GPU measurement: it runs at N = 1 only
        line["serving"] = serve_bench(gasa, args.serve_requests, local)
    if world == 1 and not args.no_other_workloads:
        # the other workloads (one warm-up and one timed solve per precision)
        with ClockSampler(local) as clk2:
            line["other_workloads"] = other_workloads(gasa, local)
        line["other_workloads_clocks"] = clk2.summary()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    del x_host
    return 0


if __name__ == "__main__":
    sys.exit(main() or 0)
