"""A plain C99 program drives the library on the GPU through include/lbm.h
alone (tests/c/abi_gpu_from_c.c): create, parameters, droplet, steps in FP32
and FP64, diagnostics and a field copied to host memory, destroy."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_runs_steps_through_the_abi(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.join(ROOT, "paper_2401_03041_gb300")
    exe = str(tmp_path / "abi_gpu_from_c")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "abi_gpu_from_c.c"),
                        "-o", exe, "-L", lib_dir, "-llbm", "-Wl,-rpath," + lib_dir, "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
