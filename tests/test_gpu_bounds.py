"""The bounds-checking build (libfemenergy_bounds.so, -DFE_DEBUG_BOUNDS), through the C ABI.

Its kernels check every index they read from memory before it addresses another buffer, and
record the first one out of range instead of using it.  Two things are checked, in a child
process that loads that library (FEMENERGY_LIBRARY), so that the session's own library is
untouched:
- the record itself: a read out of range on purpose (fe_debug_bounds_selftest, whose access
  the check keeps in bounds) is recorded with its site and index, once, and reading the
  record clears it; a read in range records nothing;
- that the checks change nothing on valid meshes: every precision's energy and gradient,
  under shuffled node ids and every node renumbering, agree with the oracle at the usual
  bars (FP64 and double-float 1e-12 / 1e-10, FP32 2e-6 / 2e-5), as do the Hessian-vector
  product and the central-difference gradient, and no kernel records an index."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import sys
import numpy as np
import torch
sys.path[:0] = [__ROOT__, __HERE__]
import oracle
from parity import check_energy, check_grad, energy_scale
from paper_2109_01158_gb300 import fem, meshgen as mg

assert fem.debug_bounds_enabled(), "the bounds-checking library was not loaded"
assert fem.debug_bounds() == (0, 0)
fem.debug_bounds_selftest(5, 4)
assert fem.debug_bounds() == (99, 5)
assert fem.debug_bounds() == (0, 0)            # reading cleared it
fem.debug_bounds_selftest(-3, 4)
assert fem.debug_bounds() == (99, -3)
fem.debug_bounds_selftest(3, 4)
assert fem.debug_bounds() == (0, 0)            # in range: nothing recorded

def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()

bars = {fem.FE_F64: (1e-12, 1e-10), fem.FE_DF64: (1e-12, 1e-10), fem.FE_F32_COMP: (2e-6, 2e-5)}
meshes = [mg.shuffle_nodes(mg.neohooke_cube3d(6), seed=3), mg.shuffle_nodes(mg.plaplace_square(12), seed=5),
          mg.neohooke_rect2d(9, 7)]
for w in meshes:
    om = oracle.OracleMesh(w)
    Jref, st, _ = om.energy(w.v, densities=True)
    gref, st2 = om.gradient_exact(w.v)
    scale = energy_scale(om, w.v)
    for order in (0, 1, 2):
        for prec, (jt, gt) in bars.items():
            gm = fem.FEMesh.from_workload(w, order=order, precisions=(prec,))
            v = dev(w.v)
            J, g = gm.energy_gradient(v)
            Je, dens = gm.energy(v, densities=True)
            assert gm.sync_status() == fem.FE_OK
            check_energy(J.item(), Jref, scale, rtol=jt)
            check_grad(g.cpu().numpy(), gref, rtol=gt)
            torch.cuda.synchronize()
            rec = fem.debug_bounds()
            assert rec == (0, 0), (w.name, order, prec, rec)
            gm.close()
    # FP64 extras: Hessian-vector product (symmetric: u.Hw = w.Hu) and the central differences
    gm = fem.FEMesh.from_workload(w, precisions=(fem.FE_F64,))
    v = dev(w.v)
    rng = np.random.default_rng(7)
    a, b = dev(rng.standard_normal(w.ndof)), dev(rng.standard_normal(w.ndof))
    ha, hb = gm.hessian_vector(v, a), gm.hessian_vector(v, b)
    s1, s2 = float(torch.dot(b, ha)), float(torch.dot(a, hb))
    assert abs(s1 - s2) <= 1e-9 * max(abs(s1), 1.0)
    gfd = gm.gradient_fd(v, 1e-6)
    assert float((gfd.cpu() - torch.from_numpy(gref)).abs().max()) <= 1e-4 * max(float(np.abs(gref).max()), 1.0)
    torch.cuda.synchronize()
    assert fem.debug_bounds() == (0, 0), (w.name, "hvp/fd")
    gm.close()
print("bounds build ok")
"""


def test_bounds_build_records_out_of_range_and_changes_nothing_in_range():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = build.build(bounds=True)
    env = dict(os.environ, FEMENERGY_LIBRARY=lib)
    code = CHILD.replace("__ROOT__", repr(ROOT)).replace("__HERE__", repr(HERE))
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, env=env,
                         cwd=ROOT)
    assert res.returncode == 0, (res.stdout[-3000:], res.stderr[-3000:])
    assert "bounds build ok" in res.stdout
