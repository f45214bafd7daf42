"""NVTX ranges around the public calls: a small injection library, loaded the way a
timeline profiler is (NVTX_INJECTION64_PATH), records the ranges the library opens and
closes.  The calls here fail their argument checks, so no device is needed; the range is
opened before the checks and closed on every return path."""
import ctypes
import os
import shutil
import subprocess
import sys

import pytest

# The injection side of the NVTX protocol, written from its documented interface: the
# loader calls InitializeInjectionNvtx2 with the export-table getter; table 1 (callbacks)
# gives the function table of module 1 (core), whose slots 9 and 11 are RangePushA and
# RangePop.
INJECTION = r"""
#include <stddef.h>
#include <stdint.h>
#include <string.h>
typedef void (*fn_t)(void);
typedef const void* (*get_table_t)(uint32_t);
typedef struct { size_t size; int (*module_table)(int, fn_t***, unsigned int*); } callbacks_t;
static char log_[8192];
static size_t used_;
static int depth_, max_depth_;
static int push_a(const char* s) {
  size_t n = strlen(s);
  if (used_ + n + 2 < sizeof log_) { memcpy(log_ + used_, s, n); used_ += n; log_[used_++] = ';'; log_[used_] = 0; }
  if (++depth_ > max_depth_) max_depth_ = depth_;
  return depth_ - 1;
}
static int pop(void) { return --depth_; }
const char* trace_log(void) { return log_; }
int trace_depth(void) { return depth_; }
int trace_max_depth(void) { return max_depth_; }
int InitializeInjectionNvtx2(get_table_t get) {
  const callbacks_t* cb = (const callbacks_t*)get(1);
  fn_t** table = 0;
  unsigned int size = 0;
  if (!cb || !cb->module_table(1, &table, &size) || size < 11 || !table[9] || !table[11]) return 0;
  *table[9] = (fn_t)push_a;
  *table[11] = (fn_t)pop;
  return 1;
}
"""


@pytest.fixture(scope="module")
def libpath():
    from paper_2109_01158_gb300 import build
    return build.build()


@pytest.fixture(scope="module")
def injection(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("nvtx")
    src, so = d / "inject.c", d / "libinject.so"
    src.write_text(INJECTION)
    subprocess.run([cc, "-shared", "-fPIC", "-O1", "-o", str(so), str(src)], check=True)
    return str(so)


def test_public_calls_open_and_close_named_ranges(libpath, injection):
    code = "\n".join([
        "import ctypes, sys",
        f"inj = ctypes.CDLL({injection!r})",   # the handle the NVTX loader gets again
        "inj.trace_log.restype = ctypes.c_char_p",
        f"lib = ctypes.CDLL({libpath!r})",
        "vp = ctypes.c_void_p",
        "lib.fe_energy.argtypes = [vp, vp, vp, vp]",
        "lib.fe_gradient_exact.argtypes = [vp, vp, vp]",
        "lib.fe_energy_gradient.argtypes = [vp, vp, vp, vp]",
        "lib.fe_batch_energy_gradient.argtypes = [vp, vp, ctypes.c_int]",
        "got = [lib.fe_energy(None, None, None, None), lib.fe_gradient_exact(None, None, None),",
        "       lib.fe_energy_gradient(None, None, None, None), lib.fe_batch_energy_gradient(None, None, 0)]",
        "print(inj.trace_log().decode())",
        "print(inj.trace_depth(), inj.trace_max_depth())",
        "sys.exit(0 if got == [1, 1, 1, 1] else 1)",
    ])
    env = dict(os.environ, NVTX_INJECTION64_PATH=injection)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120, env=env)
    assert res.returncode == 0, (res.stdout, res.stderr)
    log, depth = res.stdout.strip().splitlines()[-2:]
    assert log.split(";")[:-1] == ["fe_energy", "fe_gradient_exact", "fe_energy_gradient",
                                   "fe_batch_energy_gradient"]
    assert depth.split() == ["0", "1"]      # every range closed, none nested


def test_without_a_profiler_the_ranges_cost_nothing_visible(libpath):
    """With no injection library the same calls return their status and nothing else."""
    lib = ctypes.CDLL(libpath)
    lib.fe_energy.argtypes = [ctypes.c_void_p] * 4
    assert lib.fe_energy(None, None, None, None) == 1
