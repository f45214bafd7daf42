"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point
declared in include/femenergy.h (no compute calls: this runs on a CPU-only host)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "femenergy.h")


def declared_names():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:fe_status|int|const char\s*\*)\s+(fe_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2109_01158_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_names()
    for must in ["fe_create", "fe_destroy", "fe_mesh_upload", "fe_set_model", "fe_set_load",
                 "fe_precompute", "fe_energy", "fe_gradient_exact", "fe_energy_gradient",
                 "fe_gradient_fd", "fe_energy_gradient_host", "fe_sync_status"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_names() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s(fe_\w+)$", out, flags=re.M))
    assert set(declared_names()) <= exported


def test_library_built_for_sm103a(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_binding_names_match_abi(libpath):
    from paper_2109_01158_gb300 import fem
    for n in declared_names():
        assert hasattr(fem, n), n
    assert fem.fe_version() >= 10000


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2109_01158_gb300 import fem
    with pytest.raises(RuntimeError):
        fem._lib_saved = fem._lib
        try:
            fem._lib = None
            fem.load_library(str(tmp_path / "missing.so"))
        finally:
            fem._lib = fem._lib_saved
