"""The C-ABI library builds, loads without a GPU, and exports every entry point that
include/gv.h declares; the Python binding's struct layouts match the C compiler's."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gv.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^GV_API\s+(?:gv_status|const char \*)\s*(gv_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_04782_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("gv_create", "gv_workspace_size", "gv_render_fwd", "gv_render_bwd", "gv_render_batch_fwd",
              "gv_render_batch_bwd", "gv_autotune", "gv_graph_capture", "gv_debug_bin_sort", "gv_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2501_04782_gb300 import gv
    assert sorted(gv.EXPORTS) == declared_symbols()


def test_status_strings_without_a_gpu(lib):
    lib.gv_status_string.restype = ctypes.c_char_p
    assert lib.gv_status_string(0) == b"ok"
    assert lib.gv_status_string(2) == b"key capacity exceeded"


def test_struct_layouts_match_c(tmp_path):
    from paper_2501_04782_gb300 import gv
    prog = tmp_path / "sizes.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gv.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gv_camera), sizeof(gv_gaussians),
         sizeof(gv_gaussians_grad), sizeof(gv_frame_desc), sizeof(gv_options), offsetof(gv_frame_desc, gauss_offset),
         offsetof(gv_camera, time), offsetof(gv_options, bg), offsetof(gv_gaussians, n_ctrl),
         offsetof(gv_gaussians, sh_degree), offsetof(gv_gaussians, sh), offsetof(gv_gaussians, visible),
         offsetof(gv_gaussians_grad, camera), offsetof(gv_gaussians_grad, sh));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(gv.Camera), ctypes.sizeof(gv.Gaussians), ctypes.sizeof(gv.GaussiansGrad),
            ctypes.sizeof(gv.FrameDesc), ctypes.sizeof(gv.Options), gv.FrameDesc.gauss_offset.offset,
            gv.Camera.time.offset, gv.Options.bg.offset, gv.Gaussians.n_ctrl.offset, gv.Gaussians.sh_degree.offset,
            gv.Gaussians.sh.offset, gv.Gaussians.visible.offset, gv.GaussiansGrad.camera.offset,
            gv.GaussiansGrad.sh.offset]
    assert got == want


def test_product_path_does_not_import_the_oracle():
    """The CUDA path and its binding share no code with the oracle."""
    pkg = os.path.join(ROOT, "paper_2501_04782_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.c" not in src, f


def test_options_are_validated_on_the_host(lib):
    """gv_create checks tile shape, stage depth and background before any CUDA call, so an
    invalid option set is refused without a GPU; a valid one reaches the device query
    (GV_OK with a GPU, GV_ERR_CUDA without one)."""
    from paper_2501_04782_gb300 import gv
    lib.gv_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(gv.Options)]
    lib.gv_destroy.argtypes = [ctypes.c_void_p]

    def create(tw, th, depth, bg=(0.0, 0.0, 0.0)):
        o = gv.Options(tw, th, depth, (ctypes.c_float * 3)(*bg))
        h = ctypes.c_void_p()
        st = lib.gv_create(ctypes.byref(h), ctypes.byref(o))
        if st == 0:
            lib.gv_destroy(h)
        else:
            assert not h.value  # nothing handed out on failure
        return st

    for tw, th in ((12, 12), (8, 16), (16, 32), (64, 64), (0, 0), (-8, 8)):
        assert create(tw, th, 128) == 1, (tw, th)
    for depth in (0, 16, 48, 100, 512):
        assert create(16, 16, depth) == 1, depth
    assert create(16, 16, 128, (float("nan"), 0.0, 0.0)) == 1
    assert create(16, 16, 128, (0.0, float("inf"), 0.0)) == 1
    assert lib.gv_create(None, None) == 1
    for tw, th in ((8, 8), (16, 8), (16, 16), (32, 16), (32, 32)):
        for depth in (32, 64, 128, 256):
            assert create(tw, th, depth) in (0, 4), (tw, th, depth)
