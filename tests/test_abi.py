"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/mcrt.h declares; the Python structures match the C layout.  CPU only: no
compute call is made here."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2512_01283_gb300 import build as B
from paper_2512_01283_gb300 import mcrt as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mcrt.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^MCRT_API\s+[^;(]*?\b(mcrt_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["mcrt_create_grid", "mcrt_set_dust_tables", "mcrt_launch_packets", "mcrt_image_stokes",
                 "mcrt_destroy"]:
        assert name in syms
    assert sorted(M.SYMBOLS) == syms


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", M.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mcrt_\w+)", out))
    assert set(declared_symbols()) <= exported
    for name in declared_symbols():
        assert getattr(lib, name) is not None


def test_last_error_without_context(lib):
    assert lib.mcrt_last_error(None) is not None


def test_struct_layout_matches_c():
    """sizeof/offsetof of the public structs, compiled from the header with gcc."""
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "mcrt.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mcrt_source), sizeof(mcrt_camera),
             sizeof(mcrt_launch_desc), sizeof(mcrt_stats), offsetof(mcrt_launch_desc, pid_begin),
             offsetof(mcrt_launch_desc, time_budget_s), offsetof(mcrt_launch_desc, trace),
             offsetof(mcrt_camera, npix), sizeof(mcrt_patch), offsetof(mcrt_patch, kappa_abs));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    py = [C.sizeof(M.Source), C.sizeof(M.Camera), C.sizeof(M.LaunchDesc), C.sizeof(M.Stats),
          M.LaunchDesc.pid_begin.offset, M.LaunchDesc.time_budget_s.offset, M.LaunchDesc.trace.offset,
          M.Camera.npix.offset, C.sizeof(M.Patch), M.Patch.kappa_abs.offset]
    assert vals == py


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(M, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(M, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        M.lib()
