"""Pipelined evaluations on host buffers (fe_energy_gradient_host_async + fe_host_wait):
every result is bitwise the one of the synchronous fe_energy_gradient_host on the same v,
and matches the oracle; page-locked and pageable buffers give the same results; a domain
error in any evaluation of the sequence is reported by the wait and then cleared."""
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, check_grad, energy_scale

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _fem():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01158_gb300 import fem
    return fem


def _host(shape, pinned):
    t = torch.zeros(shape, dtype=torch.float64)
    return (t.pin_memory() if pinned else t).numpy()


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_pipelined_results_equal_the_synchronous_call(precision, pinned):
    fem = _fem()
    w = mg.shuffle_nodes(mg.random_small(17, 3, mg.MODEL_NEOHOOKE, 7, 6, 5))
    gm = fem.FEMesh.from_workload(w, order=fem.FE_ORDER_MORTON, precisions=(precision,))
    n_eval = 5
    V = _host((n_eval, w.ndof), pinned)
    for k in range(n_eval):
        V[k] = w.v + 1e-3 * mg.uniform(100 + k, np.arange(w.ndof), -1.0, 1.0)
    J = _host((n_eval, 1), pinned)
    G = _host((n_eval, w.ndof), pinned)
    for k in range(n_eval):
        gm.energy_gradient_host_async(V[k], J[k], G[k])
    assert gm.host_wait() == fem.FE_OK
    for k in range(n_eval):
        Jk, gk, st = gm.energy_gradient_host(V[k].copy())
        assert st == fem.FE_OK
        assert J[k, 0] == Jk and np.array_equal(G[k], gk), k
    om = oracle.OracleMesh(w)
    v = V[n_eval - 1].copy()
    check_energy(float(J[n_eval - 1, 0]), om.energy(v)[0], energy_scale(om, v))
    check_grad(G[n_eval - 1], om.gradient_exact(v)[0])


def test_pipelined_domain_error_is_reported_by_the_wait():
    fem = _fem()
    w = mg.neohooke_cube3d(3)
    gm = fem.FEMesh.from_workload(w)
    good = _host((w.ndof,), True)
    good[:] = w.coords.ravel()
    bad = good.copy()
    bad[3 * 21] += 2.0                      # inverts the elements around node 21
    J = _host((3, 1), True)
    G = _host((3, w.ndof), True)
    gm.energy_gradient_host_async(good, J[0], G[0])
    gm.energy_gradient_host_async(bad, J[1], G[1])
    gm.energy_gradient_host_async(good, J[2], G[2])
    assert gm.host_wait() == fem.FE_EDOMAIN
    assert J[1, 0] == math.inf and math.isfinite(J[0, 0]) and J[0, 0] == J[2, 0]
    assert np.array_equal(G[0], G[2])
    gm.energy_gradient_host_async(good, J[0], G[0])
    assert gm.host_wait() == fem.FE_OK       # status cleared by the previous wait
    with pytest.raises(ValueError):
        gm.energy_gradient_host_async(good[:-1], J[0], G[0])
