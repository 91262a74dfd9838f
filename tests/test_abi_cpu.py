"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/btrace.h declares (no GPU needed; no compute calls)."""
import ctypes as C
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "btrace.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bt_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1912_03998_gb300 import build_lib
    if not os.path.exists(build_lib.LIB) and shutil.which("nvcc") is None \
            and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build libbtrace")
    return build_lib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("bt_create", "bt_destroy", "bt_load_scene", "bt_set_sources", "bt_set_microphones",
              "bt_trace", "bt_read_levels", "bt_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_1912_03998_gb300 import btrace
    assert set(btrace.EXPECTED_SYMBOLS) == set(declared_functions())


def test_params_default_is_host_only(libpath):
    from paper_1912_03998_gb300 import btrace
    p = btrace.bt_params_default()
    assert p.max_order == 4 and abs(p.t_eps_m - 1e-3) < 1e-9
    assert p.tiles_x == 1 and p.tiles_y == 1 and p.precision == btrace.BT_PREC_MIXED
    assert list(p.air_atten_db_per_m) == [0.0] * 8 and p.count_work == 0


def test_struct_sizes_match_header(libpath):
    # the ctypes mirrors must have the C layout: 4-byte fields only in params
    from paper_1912_03998_gb300 import btrace
    assert C.sizeof(btrace.bt_trace_params) == 4 * (1 + 8 + 1 + 1 + 2 + 1 + 1 + 1 + 1 + 1 + 1 + 3)
    assert C.sizeof(btrace.bt_stats) == 8 * (14 + 3)


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    from paper_1912_03998_gb300 import btrace
    L = btrace.lib()
    assert L.bt_params_default(None) == btrace.BT_E_INVALID
    assert L.bt_destroy(None) == btrace.BT_OK
    assert L.bt_create(None, 0, None) == btrace.BT_E_INVALID
    assert L.bt_trace(None, 0, None) == btrace.BT_E_INVALID
    assert L.bt_set_result(None, 0, None, None) == btrace.BT_E_INVALID
    assert L.bt_batch_create(None, None, 0, None, None) == btrace.BT_E_INVALID
    assert L.bt_batch_run(None) == btrace.BT_E_INVALID
    assert L.bt_batch_stats(None, None) == btrace.BT_E_INVALID
    assert L.bt_batch_destroy(None) == btrace.BT_OK
    assert L.bt_scene_share(None, 0, None) == btrace.BT_E_INVALID
    assert L.bt_trace_ranges(None, 0, None, None, None, None, 0) == btrace.BT_E_INVALID
    assert L.bt_ranges_stats(None, None) == btrace.BT_E_INVALID
    assert L.bt_set_directivity(None, 0, None, 0, None) == btrace.BT_E_INVALID
    assert L.bt_beam_axes(None, 0, None) == btrace.BT_E_INVALID
    assert L.bt_submit(None, 0, None) == btrace.BT_E_INVALID
    assert L.bt_poll(None, 0) == btrace.BT_E_INVALID
    assert L.bt_wait(None, 0) == btrace.BT_E_INVALID
    assert L.bt_last_error(None) == b"null context"
    assert btrace.bt_kernel_launches() == 0


def test_plain_c_program_uses_the_boundary(libpath, tmp_path):
    # the header compiles as strict C11 and a C program links and calls the
    # library (argument checks, defaults, layouts; no compute call)
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(libpath)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", libdir, "-lbtrace",
                    "-lm", f"-Wl,-rpath,{libdir}", "-o", exe], check=True, capture_output=True, text=True)
    args = [exe] + ([] if os.path.exists("/dev/nvidia0") else ["--no-device"])
    r = subprocess.run(args, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "c_abi_check: ok" in r.stdout
