"""The C-ABI library loads and exports every entry point its header declares.

No compute call is made here (no GPU is needed): this checks the boundary
itself -- the symbols, the struct sizes the binding assumes, and that calls
with invalid arguments are rejected on the host with an error string.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs3dtr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_00395_gb300 import build, gs3dtr
    build.build()
    return gs3dtr.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    from paper_2602_00395_gb300 import gs3dtr
    assert set(gs3dtr.EXPORTED) == set(names)


STRUCTS = ["gs_params", "gs_camera", "gs_frame", "gs_probe", "gs_eps_schedule", "gs_projected", "gs_sorted",
           "gs_loss", "gs_tr_config", "gs_adam_config", "gs_batch_item"]


def test_struct_sizes_match_header_layout(tmp_path):
    """The ctypes structs have the sizes a C compiler gives the header's structs."""
    import shutil
    import subprocess
    from paper_2602_00395_gb300 import gs3dtr as G
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    body = "\n".join(f'  printf("{n} %zu\\n", sizeof({n}));' for n in STRUCTS)
    src.write_text(f'#include <stdio.h>\n#include "gs3dtr.h"\nint main(void) {{\n{body}\n  return 0;\n}}\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = dict(zip(out[0::2], map(int, out[1::2])))
    for n in STRUCTS:
        assert C.sizeof(getattr(G, n)) == got[n], n
    assert got["gs_probe"] == 32 and got["gs_camera"] == 96


def test_host_argument_checks_reject_without_touching_the_device(lib):
    from paper_2602_00395_gb300 import gs3dtr as G
    assert lib.gs_version() >= 100
    # the wait diagnostic checks its limit and status pointer on the host
    assert lib.gs_wait_check(0, C.c_void_p(16), None) == G.GS_ERR_INVALID_ARG
    assert lib.gs_wait_check((1 << 20) + 1, C.c_void_p(16), None) == G.GS_ERR_INVALID_ARG
    assert lib.gs_wait_check(100, None, None) == G.GS_ERR_INVALID_ARG
    assert b"gs_wait_check" in lib.gs_last_error()
    # null arguments are rejected before any launch
    rc = lib.gs_project(None, None, G.frame_struct(1, 8, 8), None, None, None, None)
    assert rc == G.GS_ERR_INVALID_ARG
    assert b"null" in lib.gs_last_error()
    # unsupported tile shapes give a zero workspace size
    assert lib.gs_bin_sort_workspace_size(32, G.frame_struct(1, 64, 64, 12, 16), 1000) == 0
    assert lib.gs_bin_sort_workspace_size(32, G.frame_struct(1, 64, 64, 16, 16), 1000) > 0
    assert lib.gs_bin_sort_workspace_size(32, G.frame_struct(1, 64, 64, 32, 16), 1000) > 0  # eight warps
    assert lib.gs_bin_sort_workspace_size(32, G.frame_struct(1, 64, 64, 32, 32), 1000) == 0  # sixteen: no
    assert lib.gs_raster_bwd_workspace_size(32, G.frame_struct(2, 64, 64), 3) == 0
    # a 256-byte header, then 2 views x 32 columns x 28 floats of cotangent rows
    assert lib.gs_raster_bwd_workspace_size(32, G.frame_struct(2, 64, 64), 2) == 256 + 2 * 32 * 28 * 4
    cfg = G.gs_tr_config(0.9, 0.999, 1e-12, 1e-2, 0, 0)
    x = G.gs_params(10, 32, 0, 0, 16)
    rc = lib.gs_tr_update(C.byref(x), C.byref(x), C.byref(x), C.byref(x), None, C.byref(cfg), 1, 1e-6, None,
                          None, None)
    assert rc == G.GS_ERR_INVALID_ARG  # l = 0
    sched = G.gs_eps_schedule(1e-6, 1e-8, 100)
    rc = lib.gs_tr_update_dev(C.byref(x), C.byref(x), C.byref(x), C.byref(x), None, C.byref(cfg), None,
                              C.byref(sched), None, None, None)
    assert rc == G.GS_ERR_INVALID_ARG  # no device step counter
    assert lib.gs_step_advance(None, None) == G.GS_ERR_INVALID_ARG
