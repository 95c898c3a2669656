"""The C-ABI library builds, loads and exports every entry point of include/rendermap.h.

No compute calls: these run without a GPU.
"""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rendermap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1702_06813_gb300 import build, _native
    build.build()
    return _native.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "rm_cost_grad" in names and "rm_align" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1702_06813_gb300 import _native
    assert sorted(_native.exported_symbols()) == _declared()


def test_argument_errors_without_gpu(lib):
    from paper_1702_06813_gb300 import _native as N
    assert lib.rm_map_create(None, 0, None, None, 0, None) == N.RM_EINVAL
    assert b"NULL" in lib.rm_last_error()
    h = ctypes.c_void_p()
    assert lib.rm_map_create(None, -1, None, None, 0, ctypes.byref(h)) == N.RM_EINVAL
    assert lib.rm_render_depth(None, None, 0, None, None, None, None, None) == N.RM_EINVAL
    assert lib.rm_cost(None, None, None, 0, None, None, None) == N.RM_EINVAL
    assert lib.rm_pose_retract(None, None, -1, None, None, None) == N.RM_EINVAL
    assert lib.rm_map_info(None, None, None, None) == N.RM_EINVAL
    assert lib.rm_icp_terms(None, None, None, 0, 0.1, None, None) == N.RM_EINVAL
    assert lib.rm_icp_align(None, None, None, None, None, None, None) == N.RM_EINVAL
    assert lib.rm_meshify(None, None, None, None, None, None, None, None) == N.RM_EINVAL
    assert lib.rm_dfo_align(None, None, None, None, None, None, None, None) == N.RM_EINVAL
    assert lib.rm_icp_align_batch(None, None, 1, None, None, None, None) == N.RM_EINVAL
    assert lib.rm_cost_grad_vertices(None, None, None, 1, None, None, None) == N.RM_EINVAL
    assert lib.rm_depth_blur(None, 1, None, None, 1.0, None, None) == N.RM_EINVAL
    assert lib.rm_scan_from_range(None, 10, 4.0, 0.5, None, None, None) == N.RM_EINVAL   # min > max
    assert lib.rm_scan_from_range(None, -1, 0.5, 4.0, None, None, None) == N.RM_EINVAL
    assert lib.rm_scan_from_range(None, 0, 0.5, 4.0, None, None, None) == N.RM_OK        # nothing to do
    assert lib.rm_pose_from_x(None, -1, None, None) == N.RM_EINVAL
    assert lib.rm_pose_from_x(None, 0, None, None) == N.RM_OK
    intr = N.rm_intrinsics()
    intr.width, intr.height = 8, 8
    assert lib.rm_depth_normals(ctypes.byref(intr), 1, None, None, 9.0, 0, None, None, None) == N.RM_EINVAL
    assert lib.rm_depth_normals(ctypes.byref(intr), 1, None, None, 1.0, 1, None, None, None) == N.RM_EINVAL
    assert lib.rm_depth_normals(ctypes.byref(intr), 0, None, None, 1.0, 0, None, None, None) == N.RM_OK
    assert lib.rm_depth_normals(ctypes.byref(intr), 70000, None, None, 1.0, 0, None, None, None) == N.RM_EINVAL
    import numpy as np
    buf = np.zeros(2 * 64, np.float32)
    cls = np.zeros(64, np.uint8)
    # the blur's output may not overlap its input (checked before any device work)
    assert lib.rm_depth_blur(ctypes.byref(intr), 1, buf.ctypes.data, cls.ctypes.data, 1.0,
                             buf.ctypes.data + 4 * 10, None) == N.RM_EINVAL
    assert b"overlaps" in lib.rm_last_error()
    # nor may the normals' outputs overlap an input or each other
    big = np.zeros(4 * 64 * 3, np.float32)
    assert lib.rm_depth_normals(ctypes.byref(intr), 1, buf.ctypes.data, cls.ctypes.data, 1.0, 0,
                                buf.ctypes.data + 4 * 8, None, None) == N.RM_EINVAL
    assert b"normals overlaps" in lib.rm_last_error()
    assert lib.rm_depth_normals(ctypes.byref(intr), 1, buf.ctypes.data, cls.ctypes.data, 1.0, 0,
                                big.ctypes.data, cls.ctypes.data, None) == N.RM_EINVAL
    assert b"smoothed overlaps" in lib.rm_last_error()
    assert lib.rm_depth_normals(ctypes.byref(intr), 1, buf.ctypes.data, cls.ctypes.data, 1.0, 0,
                                big.ctypes.data, big.ctypes.data + 4 * 100, None) == N.RM_EINVAL
    assert b"normals overlaps smoothed" in lib.rm_last_error()
    assert lib.rm_depth_normals(None, 1, None, None, 1.0, 0, None, None, None) == N.RM_EINVAL


def test_abi_struct_sizes_match_header():
    """The ctypes mirrors have the C layouts (checked against offsets a C compiler reports)."""
    import subprocess
    import tempfile
    from paper_1702_06813_gb300 import _native as N
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "rendermap.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rm_intrinsics),
         offsetof(rm_intrinsics, rays), sizeof(rm_scan), sizeof(rm_cost_params), sizeof(rm_cost_out),
         sizeof(rm_tuning), sizeof(rm_align_params), sizeof(rm_align_report), sizeof(rm_icp_out),
         sizeof(rm_icp_params), sizeof(rm_icp_report), offsetof(rm_icp_report, n_assoc));
  printf("%zu %zu %zu\n", sizeof(rm_meshify_params), sizeof(rm_dfo_params), sizeof(rm_dfo_report));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), c, "-o", exe],
                       check=True)
        # the header is also valid C++ (its declarations sit in an extern "C" block)
        cc = os.path.join(d, "s.cc")
        open(cc, "w").write(code)
        subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.join(ROOT, "include"),
                        cc], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(N.rm_intrinsics), N.rm_intrinsics.rays.offset, ctypes.sizeof(N.rm_scan),
            ctypes.sizeof(N.rm_cost_params), ctypes.sizeof(N.rm_cost_out), ctypes.sizeof(N.rm_tuning),
            ctypes.sizeof(N.rm_align_params), ctypes.sizeof(N.rm_align_report),
            ctypes.sizeof(N.rm_icp_out), ctypes.sizeof(N.rm_icp_params), ctypes.sizeof(N.rm_icp_report),
            N.rm_icp_report.n_assoc.offset, ctypes.sizeof(N.rm_meshify_params),
            ctypes.sizeof(N.rm_dfo_params), ctypes.sizeof(N.rm_dfo_report)]
    assert got == want
