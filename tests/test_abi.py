"""The C ABI library loads and exports every entry point that include/*.h declares; host-side argument
checks reject bad input before any CUDA call (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1908_02681_gb300 import build as pcr_build
from paper_1908_02681_gb300 import pcr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pcr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    pcr_build.build()
    return pcr.load()


def test_every_declared_symbol_is_exported(lib):
    ceil = ctypes.CDLL(pcr_build.build_ceilings())
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        target = ceil if n.startswith("pcr_ceiling_") else lib
        assert hasattr(target, n), n
    import torch
    if not torch.cuda.is_available():
        assert pcr.pcr_kernel_launch_count() == 0   # nothing launched without a GPU


def test_status_strings(lib):
    for s in range(6):
        assert pcr.pcr_status_string(s).startswith("PCR_")
    assert "unknown" in pcr.pcr_status_string(99)


def test_host_argument_checks(lib):
    out = ctypes.c_void_p()
    assert lib.pcr_create_framebuffer(0, 10, 0, ctypes.byref(out)) == pcr.PCR_ERR_INVALID_ARG
    assert "width and height" in pcr.pcr_last_error_message()
    assert lib.pcr_create_framebuffer(16385, 10, 0, ctypes.byref(out)) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_create_framebuffer(10, 10, 0x80, ctypes.byref(out)) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_create_framebuffer(10, 10, 0, None) == pcr.PCR_ERR_INVALID_ARG
    v = pcr.pcr_view()
    assert lib.pcr_render_atomicmin(None, None, 0, ctypes.byref(v), None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_clear(None, None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_resolve(None, None, 0, 0, None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_get_device_status(None, None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_destroy_framebuffer(None) == pcr.PCR_OK
    # pcr_project_points: every argument error is found on the host, before any device call
    from tests.helpers import axis_view
    good = pcr.make_view(axis_view())
    assert lib.pcr_project_points(ctypes.c_void_p(8), 4, ctypes.byref(good), 16, 16, ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None) == pcr.PCR_ERR_INVALID_ARG  # misaligned points
    assert "aligned" in pcr.pcr_last_error_message()
    assert lib.pcr_project_points(ctypes.c_void_p(16), 4, ctypes.byref(good), 0, 16, ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_project_points(ctypes.c_void_p(16), 4, ctypes.byref(good), 16, 16, None,
                                  ctypes.c_void_p(16), None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_project_points(ctypes.c_void_p(16), 4, None, 16, 16, ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_project_points(None, 0, ctypes.byref(good), 16, 16, None, None, None) == pcr.PCR_OK


def test_view_marshalling():
    from tests.helpers import axis_view
    v = axis_view(depth_mode=2)
    v.ranges = [[0.0, 10.0, 1e9], [10.0, 1e4, 1e6]]
    c = pcr.make_view(v)
    assert c.n_ranges == 2 and c.ranges[1][2] == 1e6 and c.depth_mode == 2
    assert c.view_proj[14] == -1.0 and c.near_plane == 0.5
    assert ctypes.sizeof(pcr.pcr_view) == 16 * 8 + 2 * 8 + 2 * 4 + 8 + 2 * 4 + 8 * 3 * 8


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof / offsetof of every structure the binding marshals, as gcc lays them out from include/pcr.h."""
    structs = {"pcr_view": pcr.pcr_view, "pcr_tuning": pcr.pcr_tuning, "pcr_server_config": pcr.pcr_server_config,
               "pcr_request": pcr.pcr_request, "pcr_completion": pcr.pcr_completion}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pcr.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'  printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = []
    for name, cls in structs.items():
        want.append(f"{name} size {ctypes.sizeof(cls)}")
        want += [f"{name} {f[0]} {getattr(cls, f[0]).offset}" for f in cls._fields_]
    assert got[:-1] == want


def test_server_argument_checks(lib):
    out = ctypes.c_void_p()
    cfg = pcr.pcr_server_config(0, 8, 1 << 30)
    assert lib.pcr_server_create(ctypes.byref(cfg), ctypes.byref(out)) == pcr.PCR_ERR_INVALID_ARG
    cfg = pcr.pcr_server_config(2, 257, 1 << 30)
    assert lib.pcr_server_create(ctypes.byref(cfg), ctypes.byref(out)) == pcr.PCR_ERR_INVALID_ARG
    assert "max_batch_views" in pcr.pcr_last_error_message()
    assert lib.pcr_server_create(None, ctypes.byref(out)) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_server_submit(None, None, None) == pcr.PCR_ERR_INVALID_ARG
    n = ctypes.c_int32()
    assert lib.pcr_server_poll(None, None, 0, ctypes.byref(n), 0) == pcr.PCR_ERR_INVALID_ARG
    assert lib.pcr_server_destroy(None) == pcr.PCR_OK
