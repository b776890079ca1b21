"""The C ABI library builds, loads and exports every symbol include/gasa.h
declares; the Python binding's structures match the C layouts; the binding
fails loudly without the library.  No GPU work here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gasa.h")


def _lib():
    from paper_2504_13373_gb300 import build, gasa
    if not os.path.exists(gasa.LIB_PATH):
        build.build()
    return gasa


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:gasa_status|void|const char \*|int64_t)\s*(gasa_\w+)\s*\(", src, re.M))


def test_header_declares_the_binding_exports():
    gasa = _lib()
    assert header_functions() == set(gasa.EXPORTS)


def test_library_exports_every_declared_symbol():
    gasa = _lib()
    out = subprocess.run(["nm", "-D", "--defined-only", gasa.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = header_functions() - syms
    assert not missing, missing
    L = gasa.load()
    for name in header_functions():
        getattr(L, name)


C_LAYOUT = r"""
#include <stdio.h>
#include <stddef.h>
#include "gasa.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("gasa_bsr %zu\n", sizeof(gasa_bsr));
  printf("gasa_hierarchy %zu\n", sizeof(gasa_hierarchy));
  printf("gasa_options %zu\n", sizeof(gasa_options));
  printf("gasa_setup_info %zu\n", sizeof(gasa_setup_info));
  printf("gasa_solve_info %zu\n", sizeof(gasa_solve_info));
  printf("gasa_server_stats %zu\n", sizeof(gasa_server_stats));
  P(gasa_options, gamma); P(gasa_options, seed); P(gasa_options, init_candidates);
  P(gasa_options, bulk_staging); P(gasa_options, matrix_free_levels);
  P(gasa_options, hstar); P(gasa_options, delta); P(gasa_options, tail_kib);
  P(gasa_options, grid_tail); P(gasa_options, wait_budget_s); P(gasa_options, fused_restriction);
  P(gasa_options, dense_tail_dofs); P(gasa_options, folded_smoother);
  P(gasa_setup_info, omega); P(gasa_setup_info, seconds); P(gasa_setup_info, device_bytes);
  P(gasa_bsr, val); P(gasa_bsr, on_device); P(gasa_solve_info, rel_residual);
  P(gasa_server_stats, peak_running); P(gasa_server_stats, graph_launches);
  return 0;
}
"""


def test_struct_layouts_match_c(tmp_path):
    gasa = _lib()
    src = tmp_path / "layout.c"
    src.write_text(C_LAYOUT)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.rsplit(" ", 1) for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    py = {
        "gasa_bsr": ctypes.sizeof(gasa.gasa_bsr),
        "gasa_hierarchy": ctypes.sizeof(gasa.gasa_hierarchy),
        "gasa_options": ctypes.sizeof(gasa.gasa_options),
        "gasa_setup_info": ctypes.sizeof(gasa.gasa_setup_info),
        "gasa_solve_info": ctypes.sizeof(gasa.gasa_solve_info),
        "gasa_server_stats": ctypes.sizeof(gasa.gasa_server_stats),
        "gasa_options.gamma": gasa.gasa_options.gamma.offset,
        "gasa_options.seed": gasa.gasa_options.seed.offset,
        "gasa_options.init_candidates": gasa.gasa_options.init_candidates.offset,
        "gasa_options.bulk_staging": gasa.gasa_options.bulk_staging.offset,
        "gasa_options.matrix_free_levels": gasa.gasa_options.matrix_free_levels.offset,
        "gasa_options.hstar": gasa.gasa_options.hstar.offset,
        "gasa_options.delta": gasa.gasa_options.delta.offset,
        "gasa_options.tail_kib": gasa.gasa_options.tail_kib.offset,
        "gasa_options.grid_tail": gasa.gasa_options.grid_tail.offset,
        "gasa_options.wait_budget_s": gasa.gasa_options.wait_budget_s.offset,
        "gasa_options.fused_restriction": gasa.gasa_options.fused_restriction.offset,
        "gasa_options.dense_tail_dofs": gasa.gasa_options.dense_tail_dofs.offset,
        "gasa_options.folded_smoother": gasa.gasa_options.folded_smoother.offset,
        "gasa_setup_info.omega": gasa.gasa_setup_info.omega.offset,
        "gasa_setup_info.seconds": gasa.gasa_setup_info.seconds.offset,
        "gasa_setup_info.device_bytes": gasa.gasa_setup_info.device_bytes.offset,
        "gasa_bsr.val": gasa.gasa_bsr.val.offset,
        "gasa_bsr.on_device": gasa.gasa_bsr.on_device.offset,
        "gasa_solve_info.rel_residual": gasa.gasa_solve_info.rel_residual.offset,
        "gasa_server_stats.peak_running": gasa.gasa_server_stats.peak_running.offset,
        "gasa_server_stats.graph_launches": gasa.gasa_server_stats.graph_launches.offset,
    }
    for k, v in py.items():
        assert int(got[k]) == v, k


def test_default_options():
    """Section 6's smoothing counts, and the V-cycle's launch layout: fused
    residual and restriction on, the dense bottom operator from 2,048 dofs,
    the folded level-0 smoother on, the persistent and cluster tails off."""
    gasa = _lib()
    o = gasa.gasa_default_options()
    assert (o.t_pre, o.t_post, o.q_power, o.restart) == (3, 3, 3, 30)
    assert o.fused_restriction == 1 and o.dense_tail_dofs == 2048 and o.folded_smoother == 1
    assert o.grid_tail == 0 and o.tail_kib == 0 and o.bulk_staging == 0


def test_status_strings_and_host_only_calls():
    gasa = _lib()
    assert gasa.gasa_status_string(0) == "ok"
    assert "not converged" in gasa.gasa_status_string(gasa.GASA_ERR_NOT_CONVERGED)
    assert gasa.gasa_status_string(999) == "unknown status"
    assert gasa.gasa_kernel_launches() >= 0


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_2504_13373_gb300 import gasa
    monkeypatch.setattr(gasa, "_lib", None)
    monkeypatch.setattr(gasa, "LIB_PATH", os.path.join(ROOT, "no_such_libgasa.so"))
    with pytest.raises(RuntimeError):
        gasa.load()


def test_create_without_gpu_reports_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    gasa = _lib()
    with pytest.raises(gasa.GasaError):
        gasa.gasa_create(0)


def test_single_ops_validate_before_device_work():
    gasa = _lib()
    L = gasa.load()
    # invalid sizes are rejected on the host without touching the device
    assert L.gasa_bsr_mv(7, 1, 1, 1, None, None, None, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_bsr_mv(0, -1, 1, 1, None, None, None, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_jacobi_sweep(4, 0, None, None, None, None, None, None, None, 0, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_tentative(4, 3, 9, None, None, 4, 2, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_dense_inverse(0, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    # double-single product: sizes and pointers checked on the host
    assert L.gasa_bsr_mv_ds(-1, 1, 1, None, None, None, None, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_bsr_mv_ds(4, 0, 1, None, None, None, None, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_bsr_mv_ds(4, 2, 2, None, None, None, None, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_bsr_mv_ds(0, 2, 2, None, None, None, None, None, None, None, None) == gasa.GASA_OK
    # tail query without a context
    out = (ctypes.c_int32 * 3)()
    assert L.gasa_tail_info(None, 0, out) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_setup(None, None, None, None, None, None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_solve(None, None, None, ctypes.c_double(1e-10), 0, 0, None) == gasa.GASA_ERR_INVALID_ARG
    # server calls validate before device work
    srv = ctypes.c_void_p()
    assert L.gasa_server_create(ctypes.byref(srv), 0, ctypes.c_int64(1 << 30), 3) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_server_create(ctypes.byref(srv), 0, ctypes.c_int64(0), 8) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_server_add_mesh(None, None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_server_poll(None, ctypes.c_uint64(1), None, None) == gasa.GASA_ERR_INVALID_ARG
    assert L.gasa_server_destroy(None) == gasa.GASA_OK


def test_level0_timing_program_builds(tmp_path):
    """The stand-alone level-0 kernel timing program (csrc/bench_level0.cu),
    whose build line the profile summaries quote, compiles and links against
    the library's launchers (no GPU needed to build)."""
    import shutil
    gasa = _lib()
    nvcc = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which("nvcc"):
        pytest.skip("nvcc not found")
    nvcc = nvcc if os.path.exists(nvcc) else "nvcc"
    csrc = os.path.join(ROOT, "paper_2504_13373_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I" + os.path.join(ROOT, "include"), "-I" + csrc,
                    os.path.join(csrc, "bench_level0.cu"), "-o", str(tmp_path / "bench_level0"),
                    "-L" + os.path.dirname(gasa.LIB_PATH), "-lgasa"], check=True,
                   capture_output=True)
    assert (tmp_path / "bench_level0").exists()
