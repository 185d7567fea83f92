"""Host-side checks of the C ABI: the library builds and loads, exports every
function include/gmaf.h declares, and the ctypes binding's structs have the
header's layout.  No CUDA call is made, so these run without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2511_06824_gb300 import build as gbuild
from paper_2511_06824_gb300 import gmaf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmaf.h")


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return ctypes.CDLL(gbuild.LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gmaf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gmaf_assemble", "gmaf_solve_joint", "gmaf_integrate_loads",
                     "gmaf_picard_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gmaf_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)
    assert set(gmaf.EXPORTED) == set(declared_functions())


def test_status_strings_without_gpu():
    assert gmaf.status_string(0) == "ok"
    assert "contact" in gmaf.status_string(-2)
    assert gmaf.status_string(-99) == "unknown status"


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "gmaf.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("gmaf_grid %zu\n", sizeof(gmaf_grid));
  printf("gmaf_physics %zu\n", sizeof(gmaf_physics));
  printf("gmaf_texture %zu\n", sizeof(gmaf_texture));
  printf("gmaf_state %zu\n", sizeof(gmaf_state));
  printf("gmaf_solver_opts %zu\n", sizeof(gmaf_solver_opts));
  printf("gmaf_solve_info %zu\n", sizeof(gmaf_solve_info));
  printf("gmaf_request %zu\n", sizeof(gmaf_request));
  printf("gmaf_result %zu\n", sizeof(gmaf_result));
  P(gmaf_request, state) P(gmaf_request, dt) P(gmaf_request, max_iter)
  P(gmaf_result, state) P(gmaf_result, J) P(gmaf_result, G) P(gmaf_result, tile_rows)
  P(gmaf_texture, radius) P(gmaf_texture, offset_z) P(gmaf_state, edot)
  P(gmaf_solver_opts, omega) P(gmaf_solver_opts, eps) P(gmaf_solver_opts, max_iter)
  P(gmaf_solver_opts, precision) P(gmaf_solver_opts, zero_init) P(gmaf_solver_opts, criterion)
  P(gmaf_solve_info, rel_residual) P(gmaf_solve_info, true_rel_residual)
  P(gmaf_solve_info, kernel_variant) P(gmaf_solve_info, tasks) P(gmaf_solve_info, iterations_sum)
  P(gmaf_solve_info, p_update_period)
  P(gmaf_physics, p_case)
  return 0;
}
"""


def test_ctypes_structs_match_header(tmp_path):
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text(_LAYOUT_C)
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run(
        [str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for name in ("gmaf_grid", "gmaf_physics", "gmaf_texture", "gmaf_state", "gmaf_solver_opts",
                 "gmaf_solve_info", "gmaf_request", "gmaf_result"):
        assert int(got[name]) == ctypes.sizeof(getattr(gmaf, name)), name
    for key, v in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(gmaf, t), f).offset == int(v), key


def test_binding_refuses_host_arrays_for_device_arguments():
    import numpy as np
    with pytest.raises(TypeError):
        gmaf._dev(np.zeros(4), 4, "D")
