"""The library used from plain C on the GPU: tests/c_abi_check.c traces one
source over a ground plane through the C ABI alone (synchronous and
submitted) and checks every microphone against the direct-plus-image closed
form."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_traces_a_ground_plane(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_1912_03998_gb300 import build_lib
    lib = build_lib.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_check")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", libdir, "-lbtrace", "-lm",
                    f"-Wl,-rpath,{libdir}", "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe, "--trace"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c_abi_check: ok" in r.stdout
