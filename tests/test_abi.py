"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/lbm.h declares; host-side validation runs without CUDA calls."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.stencils import stencil as ostencil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2401_03041_gb300 import build, lbm
    build.build()
    return lbm.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    from paper_2401_03041_gb300 import lbm
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lbm.SYMBOLS) == names


@pytest.mark.parametrize("Q", [7, 15, 19, 27])
def test_library_stencils_match_appendix_b(L, Q):
    from paper_2401_03041_gb300 import lbm
    c, w = lbm.stencil(Q)
    S = ostencil(Q)
    assert sorted(c) == sorted(tuple(int(v) for v in r) for r in S.c)
    for ci, wi in zip(c, w):
        j = next(j for j in range(Q) if tuple(int(v) for v in S.c[j]) == ci)
        assert wi == S.w[j]


def _padded(nx, ny, nz, s):
    """Elements per direction of a PDF array with the periodic ghost cells:
    16 / s columns and 2 rows on each side, rows padded to 16 bytes."""
    gx = 16 // s
    nxp = -(-(nx + 2 * gx) // gx) * gx
    return nz * (ny + 4) * nxp


def test_workspace_bytes(L):
    nb = L.lbm_workspace_bytes(32, 32, 32, 0, 0, 15)
    pdf = 2 * (15 + 27 + 7) * _padded(32, 32, 32, 8) * 8
    assert pdf <= nb < pdf + 4 * 1024 * 1024
    nb32 = L.lbm_workspace_bytes(512, 512, 512, 1, 0, 15)
    pdf32 = 2 * 49 * _padded(512, 512, 512, 4) * 4
    assert pdf32 <= nb32 < pdf32 + 64 * 1024 * 1024
    assert pdf32 < 1.03 * 2 * 49 * 512 ** 3 * 4        # ghost cells cost < 3 %
    nb16 = L.lbm_workspace_bytes(64, 64, 64, 2, 4, 27)
    assert nb16 >= 2 * (27 + 27) * _padded(64, 64, 64, 2) * 2 + 5 * 64 ** 3 * 4
    assert L.lbm_workspace_bytes(1, 262140, 1, 1, 0, 15) > 0
    for bad in [(0, 4, 4, 0, 0, 15), (4, 4, 4, 3, 0, 15), (4, 4, 4, 0, 6, 15), (4, 4, 4, 0, 0, 19),
                (1, 262141, 1, 1, 0, 15), (1, 1, 65536, 1, 0, 15)]:
        assert L.lbm_workspace_bytes(*bad) == 0


def test_create_rejects_bad_arguments_without_cuda(L):
    h = ctypes.c_void_p()
    assert L.lbm_create_domain(0, 4, 4, 0, 0, 15, None, None, 0, ctypes.byref(h)) == -1
    assert b"invalid" in L.lbm_last_error()
    assert L.lbm_create_domain(4, 4, 4, 0, 0, 14, None, None, 0, ctypes.byref(h)) == -1
    assert L.lbm_create_domain(4, 4, 4, 0, 0, 15, None, ctypes.c_void_p(0x1000), 16,
                               ctypes.byref(h)) == -3
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_set_params(None, None) == -1
    assert L.lbm_stencil(9, None, None) == -1


def test_params_roundtrip(L):
    from paper_2401_03041_gb300 import lbm
    import workloads as W
    p = lbm.make_params(W.config2().params)
    assert p.walls_z == 1 and p.T_top == 0.5 and p.nu_L == 0.05
    assert p.omega_high == 1.0 and p.eps_n == 1e-12


def test_header_is_plain_c_and_usable_from_c(L, tmp_path):
    """include/lbm.h compiles as strict C99 and a C program linked against
    liblbm.so runs the entry points that need no GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.join(ROOT, "paper_2401_03041_gb300")
    exe = str(tmp_path / "abi_from_c")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_from_c.c"),
                        "-o", exe, "-L", lib_dir, "-llbm", "-Wl,-rpath," + lib_dir, "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_in_place_layout_workspace_about_half():
    """lbm_workspace_bytes_layout: the in-place (AA) layout holds one PDF set
    plus a (phi, T) field, about half the two-grid workspace; the plain call
    is the two-grid layout; an unknown layout gives 0."""
    from paper_2401_03041_gb300 import lbm
    L = lbm.lib()
    for prec in (0, 1, 2):
        two = L.lbm_workspace_bytes_layout(256, 256, 256, prec, 0, 15, 0)
        aa = L.lbm_workspace_bytes_layout(256, 256, 256, prec, 0, 15, 1)
        assert two == L.lbm_workspace_bytes(256, 256, 256, prec, 0, 15)
        assert 0.45 * two < aa < 0.6 * two, (prec, aa / two)
    assert L.lbm_workspace_bytes_layout(8, 8, 8, 1, 0, 15, 7) == 0
