"""The boundary from plain C: tests/c/host_call.c includes only include/femenergy.h, links
only libfemenergy.so, and evaluates J and the exact gradient through fe_energy_gradient_host
(host buffers).  CPU: it compiles against the header.  GPU: its results match the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, check_grad, energy_scale

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "host_call.c")
PKG = os.path.join(ROOT, "paper_2109_01158_gb300")


def _compile(out, link=True):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC, "-o", out]
    if link:
        cmd += ["-L", PKG, "-lfemenergy", "-Wl,-rpath," + PKG]
    else:
        cmd = cmd[:-2] + ["-c", "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def test_c_caller_compiles_against_the_header(tmp_path):
    _compile(str(tmp_path / "host_call.o"), link=False)


def _write_input(path, w):
    with open(path, "wb") as fh:
        np.array([w.dim, w.d, w.nn, w.ne, w.model], dtype=np.int64).tofile(fh)
        np.array([w.p, w.C1, w.D1], dtype=np.float64).tofile(fh)
        np.ascontiguousarray(w.coords, dtype=np.float64).tofile(fh)
        np.ascontiguousarray(w.elems, dtype=np.int32).tofile(fh)
        np.ascontiguousarray(w.dirichlet, dtype=np.uint8).tofile(fh)
        f = w.f if w.f is not None else np.zeros(w.ndof)
        np.ascontiguousarray(f, dtype=np.float64).tofile(fh)
        np.ascontiguousarray(w.v, dtype=np.float64).tofile(fh)


@pytest.mark.gpu
@pytest.mark.parametrize("maker", [lambda: mg.random_small(91, 3, mg.MODEL_NEOHOOKE, 6, 5, 4),
                                   lambda: mg.plaplace_square(32, p=3.0)])
def test_c_caller_matches_oracle(tmp_path, maker):
    from paper_2109_01158_gb300 import build
    build.build()
    exe = str(tmp_path / "host_call")
    _compile(exe)
    w = maker()
    _write_input(str(tmp_path / "in.bin"), w)
    res = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    raw = np.fromfile(str(tmp_path / "out.bin"), dtype=np.uint8)
    st = int(raw[:8].view(np.int64)[0])
    J = float(raw[8:16].view(np.float64)[0])
    g = raw[16:].view(np.float64)
    assert st == 0 and g.size == w.ndof
    om = oracle.OracleMesh(w)
    check_energy(J, om.energy(w.v)[0], energy_scale(om, w.v))
    check_grad(g, om.gradient_exact(w.v)[0])
