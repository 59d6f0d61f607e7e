"""Host-side guards of the C-ABI that need no GPU.

* The fused kernel for a tile_x x tile_y tile stages TMA boxes whose sizes are
  encoded in the board's tensor maps; a plan whose tile differs from the
  maps' is refused (FDTD_EINVAL) before anything is launched.  The check is
  the header function the plan build calls (``fused_maps_match`` in
  csrc/fdtd_internal.h), compiled here into a small host program with forced
  mismatches.
* Storage precisions other than FP32 and FP16 are refused by fdtd_create
  before any device work.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1008_2602_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "fdtd_internal.h"
using namespace fdtd;
int main()
{
    static CUtensorMap maps[kNumMaps];
    Board h{};
    h.ix0 = 12; h.ix1 = 868; h.iy0 = 12; h.iy1 = 668;   // a board with a fused region
    h.tm = maps; h.tm_tx = 62; h.tm_ty = 8;
    int bad = 0;
    bad += !fused_maps_match(h, 62, 8);      // the tile the maps were encoded for
    bad += fused_maps_match(h, 62, 4);       // fewer rows: boxes would overrun the stage
    bad += fused_maps_match(h, 124, 8);      // wider tile
    bad += fused_maps_match(h, 124, 4);
    h.tm = nullptr;
    bad += fused_maps_match(h, 62, 8);       // maps never encoded
    Board e{};                                // no fused region: nothing to match
    e.ix0 = e.ix1 = 0;
    bad += !fused_maps_match(e, 124, 4);
    std::printf("%d\n", bad);
    return bad;
}
"""


def test_plan_build_refuses_a_tile_that_does_not_match_the_tensor_maps(tmp_path):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda.h")):
        pytest.skip("g++ and the CUDA headers are needed to compile the host check")
    src = tmp_path / "guard.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "guard"
    subprocess.run([gxx, "-std=c++17", "-I", CSRC, "-I", cuda_inc, "-o", str(exe), str(src)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "0", r.stdout


def test_retired_and_unknown_precisions_are_refused_before_device_work():
    from paper_1008_2602_gb300 import capi
    g = capi.fdtd_grid(4, 4, 4, 1e-3, 1e-3, 1e-3, 0.99, 0.0)
    b = capi.fdtd_boundary((ctypes.c_int * 6)(*([0] * 6)), 3.0, 1e-6, 1.0, (ctypes.c_int * 6)(*([0] * 6)))
    mat = np.zeros((4, 4, 4), np.uint8)
    eps = np.ones(1)
    ctx = ctypes.c_void_p()
    for prec in (2, 3, -1):
        rc = capi.lib.fdtd_create(ctypes.byref(g), mat.ctypes.data_as(ctypes.c_void_p),
                                  eps.ctypes.data_as(ctypes.c_void_p), 1, None, 0, None, ctypes.byref(b), prec,
                                  None, ctypes.byref(ctx))
        assert rc == capi.FDTD_EINVAL, prec
        assert "FP32" in capi.lib.fdtd_last_error().decode()
