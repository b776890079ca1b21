"""The benchmark's algorithmic-byte model of one CG iteration (the whole
iteration roofline), on a two-level hierarchy small enough to count by hand:
2 units of 2 dofs with 4 blocks on level 0, 1 coarse unit of 1 dof, 3 + 3
smoothing steps, FP32 words."""
import bench

LEVEL0 = {"units": 2, "s": 2, "nnzb": 4, "R_nnzb": 2, "P_nnzb": 2, "s_next": 1, "RA_nnzb": 0}
COARSE = {"units": 1, "s": 1, "nnzb": 1, "R_nnzb": 0, "P_nnzb": 0, "s_next": 0, "RA_nnzb": 0}

# level 0 by hand: |A| = 4*4*4 + 4*4 + 4*3 = 92, |W| = 2*4*4 = 32, a vector 2*2*4 = 16,
# |R| = 2*2*4 + 2*4 + 2*4 = 32, |P| = 2*2*4 + 2*4 + 3*4 = 36, the coarse vector 4
FIRST = 32 + 4 * 16          # W, the FP64 residual read, x and its FP32 copy written
RESID = 92 + 3 * 16
RESTRICT = 32 + 16 + 4
PROLONG = 36 + 4 + 2 * 16


def parts(folded, precision="mixed32"):
    shapes = [dict(LEVEL0, folded=folded), dict(COARSE)]
    return bench.iteration_bytes(shapes, precision, 3, 3)[1]


def test_plain_level0_steps():
    p = parts(False)
    assert p["level0"] == FIRST + 5 * (92 + 32 + 3 * 16) + RESID + RESTRICT + PROLONG
    assert p["coarse"] == 1 * 8 + 2 * 4


def test_folded_level0_steps_read_wa_and_c_not_a_w_and_b():
    """u + c - (W A) u: each of the five later steps reads W A (the size of A),
    c, u and writes the result; the first step also writes c."""
    p = parts(True)
    assert p["level0"] == (FIRST + 16) + 5 * (92 + 3 * 16) + RESID + RESTRICT + PROLONG
    assert parts(False)["level0"] - p["level0"] == 5 * 32 - 16


def test_fp16_and_fp64_cycles_keep_the_plain_step():
    for prec in ("mixed16", "fp64"):
        assert parts(True, prec)["level0"] == parts(False, prec)["level0"]


def test_dense_bottom_replaces_the_levels_below():
    """With the dense operator from level 1, level 1's steps and the coarsest
    solve become one n_1 x n_1 product (8 bytes per entry) and its two vectors."""
    mid = {"units": 2, "s": 1, "nnzb": 4, "R_nnzb": 2, "P_nnzb": 2, "s_next": 1, "RA_nnzb": 0}
    shapes = [dict(LEVEL0, s_next=1, units=2), dict(mid, dense_tail=True), dict(COARSE)]
    p = bench.iteration_bytes(shapes, "mixed32", 3, 3)[1]
    assert "level1" not in p and "coarse" not in p
    assert p["dense_tail"] == 2 * 2 * 8 + 2 * 2 * 4


def test_clock_summary_uses_samples_under_load():
    """The clock record's SM clock is the median of the samples taken under
    load; idle samples between launches do not pull it down, throttle
    reasons seen in any sample are reported, malformed lines are skipped."""
    import bench
    lines = [
        "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active, 100",
        "2055, 2070, 950.3, Not Active, Not Active, Not Active, Active, 98",
        "2070, 2070, 940.0, Not Active, Not Active, Not Active, Not Active, 99",
        "345, 2070, 120.0, Not Active, Not Active, Not Active, Not Active, 0",
        "210, 2070, 110.0, Not Active, Not Active, Not Active, Not Active, 3",
        "[N/A], 2070, 100.0, Not Active, Not Active, Not Active, Not Active, 0",
        "garbage",
    ]
    out = bench.ClockSampler.parse(lines)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["samples"] == 5 and out["samples_under_load"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.ClockSampler.parse(["1500, 2070, 1300, Active, Not Active, Not Active, Not Active, 100"])
    assert hot["reasons"] == ["hw_slowdown"] and hot["sm_mhz"] == 1500.0
    # without a utilisation column every sample counts
    old = bench.ClockSampler.parse(["2000, 2070, 900, Not Active, Not Active, Not Active, Not Active",
                                    "1000, 2070, 900, Not Active, Not Active, Not Active, Not Active"])
    assert old["sm_mhz"] == 1500.0 and old["samples_under_load"] == 0
    assert bench.ClockSampler.parse([])["reasons"] == ["no samples"]
