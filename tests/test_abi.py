"""The C-ABI library loads and exports every entry point its header declares
(no GPU needed: nothing here launches a kernel), and host-side argument checks
answer before any device work."""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "arbx.h"
LIB = ROOT / "paper_2507_23700_b300" / "libarbx.so"
LIB_CHECKED = ROOT / "paper_2507_23700_b300" / "libarbx_checked.so"


def declared_functions() -> list[str]:
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(arbx_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not LIB.exists():
        from paper_2507_23700_b300 import _build  # noqa: F401  (import error if package broken)
        pytest.fail("libarbx.so is not built; run python paper_2507_23700_b300/_build.py")
    return ctypes.CDLL(str(LIB))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["arbx_build", "arbx_tree_info", "arbx_tree_destroy", "arbx_query_crs", "arbx_crs_free",
                     "arbx_query_callback", "arbx_query_knn", "arbx_query_ray_nearest", "arbx_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_library_exports_the_same_boundary(lib):
    """The bounds-checked build has every entry point, says so, and keeps the
    ABI version and the host-side argument checks."""
    if not LIB_CHECKED.exists():
        pytest.fail("libarbx_checked.so is not built; run python paper_2507_23700_b300/_build.py --checked")
    chk = ctypes.CDLL(str(LIB_CHECKED))
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing
    chk.arbx_library_flags.restype = ctypes.c_uint32
    lib.arbx_library_flags.restype = ctypes.c_uint32
    assert chk.arbx_library_flags() == 1 and lib.arbx_library_flags() == 0
    assert chk.arbx_abi_version() == lib.arbx_abi_version()
    chk.arbx_status_string.restype = ctypes.c_char_p
    assert b"range" in chk.arbx_status_string(9)
    assert chk.arbx_build(None, None, None) == 1


def test_binding_covers_every_declared_symbol():
    import paper_2507_23700_b300 as arbx
    assert set(declared_functions()) <= set(arbx.exported_symbols())


def test_status_strings(lib):
    lib.arbx_status_string.restype = ctypes.c_char_p
    assert lib.arbx_status_string(0) == b"ok"
    assert b"invalid" in lib.arbx_status_string(1)
    assert lib.arbx_abi_version() == 3


def test_host_argument_checks_need_no_device(lib):
    import paper_2507_23700_b300 as arbx
    h = ctypes.c_void_p()
    assert lib.arbx_build(None, None, None) == arbx.ERR_INVALID
    bad = arbx.arbx_primitives(arbx.POINT, 3, -1, None, 0)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(bad), None) == arbx.ERR_INVALID
    nodata = arbx.arbx_primitives(arbx.POINT, 3, 10, None, 0)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(nodata), None) == arbx.ERR_INVALID
    baddim = arbx.arbx_primitives(arbx.POINT, 11, 10, 1234, 0)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(baddim), None) == arbx.ERR_INVALID
    tri2d = arbx.arbx_primitives(arbx.TRIANGLE, 2, 10, 1234, 0)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(tri2d), None) == arbx.ERR_INVALID
    q_points = arbx.arbx_primitives(arbx.POINT, 3, 10, 1234, arbx.QUANTIZED_NODES)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(q_points), None) == arbx.ERR_UNSUPPORTED
    w_tris = arbx.arbx_primitives(arbx.TRIANGLE, 3, 10, 1234, arbx.WIDE_NODES)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(w_tris), None) == arbx.ERR_UNSUPPORTED
    bad_flag = arbx.arbx_primitives(arbx.POINT, 3, 10, 1234, 8)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(bad_flag), None) == arbx.ERR_INVALID
    # the parent-relative form is a variant of the 16-bit nodes, for triangles
    p_alone = arbx.arbx_primitives(arbx.TRIANGLE, 3, 10, 1234, arbx.PARENT_RELATIVE)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(p_alone), None) == arbx.ERR_INVALID
    p_points = arbx.arbx_primitives(arbx.POINT, 3, 10, 1234, arbx.QUANTIZED_NODES | arbx.PARENT_RELATIVE)
    assert lib.arbx_build(ctypes.byref(h), ctypes.byref(p_points), None) == arbx.ERR_UNSUPPORTED
    assert lib.arbx_tree_info(None, None, None, None) == arbx.ERR_INVALID
    assert lib.arbx_tree_destroy(None) == arbx.OK
    assert lib.arbx_query_crs(None, None, 0, None, None, None) == arbx.ERR_INVALID


def test_no_launches_without_work():
    import paper_2507_23700_b300 as arbx
    assert arbx.launch_count() == 0


def test_autotune_records_round_trip(tmp_path):
    """Recorded launch settings survive save -> clear -> load; lines with an
    invalid setting are dropped (no device work: the records are host state)."""
    import paper_2507_23700_b300 as arbx
    src = tmp_path / "tune_in.txt"
    src.write_text("# comment\n"
                   "NVIDIA_B300 0 3 0 23 10 0 128 1 255 0 0 1\n"        # 13 fields: lanes default
                   "NVIDIA_B300 2 3 8 23 10 0 256 0 0 0 1 0 4\n"
                   "NVIDIA_B300 2 3 16 23 10 0 256 0 0 0 1 0 3\n"   # lanes not 1/2/4/8/16/32
                   "NVIDIA_B300 2 3 8 23 11 0 256 0 0 0 1 0 1 0\n"  # 15 fields: binary nodes
                   "NVIDIA_B300 2 3 8 23 12 0 256 0 0 0 1 0 1 2\n"  # wide_nodes not -1/0/1
                   "NVIDIA_B300 2 3 1 23 13 0 256 1 0 0 0 0 1 0 1\n"  # 16 fields: warp packets
                   "NVIDIA_B300 2 3 16 23 14 0 256 1 0 0 0 0 1 0 0 4\n"  # 17 fields: lane runs of 4
                   "NVIDIA_B300 2 3 16 23 15 0 256 1 0 0 0 0 1 0 0 3\n"  # runs not 1/4/8
                   "NVIDIA_B300 0 3 0 20 5 0 100 1 255 0 0 0\n"      # block not a multiple of 32
                   "NVIDIA_B300 0 3 0 20 6 0 128 1 77 0 0 0\n"       # top levels not 0/255/1023
                   "NVIDIA_B300 0 3 0 20 7 0 128 1 255 0 0\n")       # a field missing
    arbx.autotune_clear()
    arbx.autotune_load(src)
    out = tmp_path / "tune_out.txt"
    arbx.autotune_save(out)
    lines = [ln for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert lines == ["NVIDIA_B300 0 3 0 23 10 0 128 1 255 0 0 1 0 -1 -1 0",
                     "NVIDIA_B300 2 3 1 23 13 0 256 1 0 0 0 0 1 0 1 0",
                     "NVIDIA_B300 2 3 8 23 10 0 256 0 0 0 1 0 4 -1 -1 0",
                     "NVIDIA_B300 2 3 8 23 11 0 256 0 0 0 1 0 1 0 -1 0",
                     "NVIDIA_B300 2 3 16 23 14 0 256 1 0 0 0 0 1 0 0 4"]
    arbx.autotune_clear()
    arbx.autotune_save(out)
    assert [ln for ln in out.read_text().splitlines() if not ln.startswith("#")] == []
    with pytest.raises(arbx.ArbxError):
        arbx.autotune_load(tmp_path / "missing.txt")


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as strict C99 (no C++ or torch types), and
    a C program links against the library's exports."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "arbx.h"\n'
                   '#include <stdio.h>\n'
                   'int main(void) {\n'
                   '  arbx_tuning t = {0, -1, -1, 0, -1, -1, -1, 0, -1, -1, 0};\n'
                   '  arbx_predicates p = {ARBX_RAY_ORDERED, 3, 0, 0, 0, 0.0f, 0, 0};\n'
                   '  (void)t; (void)p;\n'
                   '  printf("%zu %zu %zu %zu %zu\\n", sizeof(arbx_tuning), sizeof(arbx_predicates),\n'
                   '         sizeof(arbx_primitives), sizeof(arbx_crs), sizeof(arbx_request));\n'
                   '  return arbx_abi_version() == 3 ? 0 : 1;\n'
                   '}\n')
    exe = tmp_path / "use"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", f"-I{ROOT / 'include'}",
                        str(src), str(LIB), f"-Wl,-rpath,{LIB.parent}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0
    # the binding's ctypes structs have the C layout
    import paper_2507_23700_b300 as arbx
    sizes = [int(x) for x in run.stdout.split()]
    assert sizes == [ctypes.sizeof(c) for c in (arbx.arbx_tuning, arbx.arbx_predicates, arbx.arbx_primitives,
                                                arbx.arbx_crs, arbx.arbx_request)]
