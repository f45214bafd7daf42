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


def _compile(out, link=True, src=SRC):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src, "-o", out]
    if link:
        cmd += ["-L", PKG, "-lfemenergy", "-Wl,-rpath," + PKG]
    else:
        cmd = cmd[:-2] + ["-c", "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def test_c_caller_compiles_against_the_header(tmp_path):
    _compile(str(tmp_path / "host_call.o"), link=False)


def test_c_caller_of_the_host_side_node_order(tmp_path):
    """tests/c/node_order.c links libfemenergy.so and calls fe_node_order, which needs no
    device.  The strip is numbered row by row, so its natural bandwidth is n + 2.  Reverse
    Cuthill-McKee brings it to 2, the least any numbering of the strip has.  The Morton
    curve, on one scale for both axes, keeps neighbours a few indices apart."""
    from paper_2109_01158_gb300 import build
    if not os.path.exists(os.path.join(PKG, "libfemenergy.so")):
        build.build()
    exe = str(tmp_path / "node_order")
    _compile(exe, src=os.path.join(ROOT, "tests", "c", "node_order.c"))
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    bw = dict(line.split()[1::2] for line in res.stdout.splitlines())
    assert bw["0"] == "42" and bw["2"] == "2" and int(bw["1"]) < 8


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
