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
    """Every translation unit is compiled with one -gencode, for sm_103a only."""
    from paper_2109_01158_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getmtime(libpath) >= max(os.path.getmtime(os.path.join(build.CSRC, f))
                                            for f in os.listdir(build.CSRC) if f.endswith((".cu", ".cuh", ".h")))


# Every entry point whose first argument is the context, with the number of arguments after it.
_CTX_CALLS = {
    "fe_destroy": 0, "fe_set_stream": 1, "fe_mesh_upload": 8, "fe_set_model": 4, "fe_set_load": 1,
    "fe_precompute": 1, "fe_set_precision": 1, "fe_set_input": 1, "fe_set_vector_order": 1,
    "fe_to_device_order": 2, "fe_from_device_order": 2, "fe_footprint": 1, "fe_energy": 3,
    "fe_gradient_exact": 2, "fe_energy_gradient": 3, "fe_hessian_vector": 3, "fe_cg_steihaug": 9,
    "fe_gradient_fd": 5, "fe_energy_gradient_host": 3, "fe_energy_gradient_host_async": 3, "fe_host_wait": 0,
    "fe_sync_status": 0, "fe_set_wait_limit": 1, "fe_get_shape_gradients": 2, "fe_get_patches": 2, "fe_get_load_vector": 1,
}


def test_null_context_is_rejected(libpath):
    """Each call on a NULL context returns FE_EINVAL (fe_destroy: FE_OK) without touching the
    device.  Run in a child process, so that a crash fails the test instead of the session."""
    code = "\n".join([
        "import ctypes, sys",
        f"lib = ctypes.CDLL({libpath!r})",
        "bad = []",
        f"for name, n in {_CTX_CALLS!r}.items():",
        "    fn = getattr(lib, name)",
        "    fn.restype = ctypes.c_int",
        "    fn.argtypes = [ctypes.c_void_p] * (n + 1)",
        "    st = fn(*([None] * (n + 1)))",
        "    want = 0 if name == 'fe_destroy' else 1",
        "    if st != want: bad.append((name, st))",
        "print(bad)",
        "sys.exit(1 if bad else 0)",
    ])
    import sys
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, (res.stdout, res.stderr)


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


def test_device_free_argument_checks(libpath):
    """Argument checks that come before any device call: the FP64 rate probe with an unknown
    operation or a null result pointer, a batch executor's negative wait limit on a null
    handle.  Run in a child process, so that a crash fails the test instead of the session."""
    code = "\n".join([
        "import ctypes, sys",
        f"lib = ctypes.CDLL({libpath!r})",
        "lib.fe_fp64_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]",
        "lib.fe_batch_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_int64]",
        "r = ctypes.c_double()",
        "got = [lib.fe_fp64_rate(0, 3, ctypes.byref(r), None), lib.fe_fp64_rate(0, -1, ctypes.byref(r), None),",
        "       lib.fe_fp64_rate(0, 0, None, None), lib.fe_batch_set_wait_limit(None, 5)]",
        "print(got)",
        "sys.exit(0 if got == [1, 1, 1, 1] else 1)",
    ])
    import sys
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, (res.stdout, res.stderr)


def test_bounds_calls_in_the_ordinary_build(libpath):
    """The ordinary build reports that its kernels are not bounds-checked: no record, and the
    self-test refused (its read would not be checked).  No device call is made."""
    code = "\n".join([
        "import ctypes, sys",
        f"lib = ctypes.CDLL({libpath!r})",
        "lib.fe_debug_bounds.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]",
        "lib.fe_debug_bounds_selftest.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64]",
        "site, index = ctypes.c_int(7), ctypes.c_int64(7)",
        "got = [lib.fe_debug_bounds_enabled(), lib.fe_debug_bounds(0, ctypes.byref(site), ctypes.byref(index)),",
        "       site.value, index.value, lib.fe_debug_bounds_selftest(0, 5, 4), lib.fe_debug_bounds(0, None, None)]",
        "print(got)",
        "sys.exit(0 if got == [0, 0, 0, 0, 1, 1] else 1)",
    ])
    import sys
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, (res.stdout, res.stderr)


def test_bounds_checking_build_links_and_exports_the_boundary():
    """The bounds-checking variant (-DFE_DEBUG_BOUNDS) builds, says so, and exports every
    symbol the header declares (loading it registers the kernels' error words; no device call)."""
    from paper_2109_01158_gb300 import build
    lib_path = build.build(bounds=True)
    assert lib_path != build.LIB
    code = "\n".join([
        "import ctypes, sys",
        f"lib = ctypes.CDLL({lib_path!r})",
        f"names = {declared_names()!r}",
        "missing = [n for n in names if not hasattr(lib, n)]",
        "print(missing, lib.fe_debug_bounds_enabled())",
        "sys.exit(0 if not missing and lib.fe_debug_bounds_enabled() == 1 else 1)",
    ])
    import sys
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, (res.stdout, res.stderr)
