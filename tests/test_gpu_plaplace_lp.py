"""The componentwise p-Laplacian (FE_PLAPLACE_LP) on the GPU: energy, exact gradient,
central-difference gradient and Hessian-vector product against the oracle, the calls that
reject it, and the Benchmark 6 minima reached by trust-region Newton-CG on the FP64 kernels."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, check_grad, energy_scale, fd_extra

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _fem():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01158_gb300 import fem
    return fem


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("seed,dim,p,n", [(41, 2, 3.0, (17, 13)), (42, 2, 1.5, (9, 11)), (43, 3, 4.5, (6, 5, 4)),
                                          (44, 2, 2.0, (8, 8))])
@pytest.mark.parametrize("order", [0, 1])
def test_componentwise_plaplace_matches_oracle(seed, dim, p, n, order):
    fem = _fem()
    w = mg.random_small(seed, dim, mg.MODEL_PLAPLACE, *n, p=p)
    w.model = mg.MODEL_PLAPLACE_LP
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w, order=order)
    v = _dev(w.v)
    J, g = gm.energy_gradient(v)
    assert gm.sync_status() == fem.FE_OK
    check_energy(J.item(), om.energy(w.v)[0], energy_scale(om, w.v))
    check_grad(g.cpu().numpy(), om.gradient_exact(w.v)[0])
    check_grad(gm.gradient_fd(v, 1e-6).cpu().numpy(), om.gradient_fd(w.v, 1e-6)[0],
               extra_abs=fd_extra(om, w.v, 1e-6))
    x = mg.uniform(seed + 1, np.arange(w.ndof), -1.0, 1.0)
    check_grad(gm.hessian_vector(v, _dev(x)).cpu().numpy(), om.hessian_vector(w.v, x)[0])


def test_componentwise_plaplace_is_fp64_only():
    fem = _fem()
    w = mg.plaplace_square(8, p=3.0)
    w.model = mg.MODEL_PLAPLACE_LP
    gm = fem.FEMesh.from_workload(w, precisions=(fem.FE_DF64, fem.FE_F64))
    with pytest.raises(fem.FEError):
        gm.energy(_dev(w.v))
    gm.set_precision(fem.FE_F64)
    gm.energy(_dev(w.v))
    srv = fem.NativeServer(0, 1 << 26, 4)
    with pytest.raises(fem.FEError):
        srv.submit(gm, w.v.copy(), np.zeros(1), np.zeros(gm.ndof))
    srv.close()


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5, 6])
def test_gpu_benchmark6_minimal_energies(level):
    """Benchmark 6 on the FP64 kernels: trust-region Newton-CG from v = 0 reaches the printed
    J(u) of every level up to 6 (48,641 free dofs) to its 4 decimals."""
    fem = _fem()
    from paper_2109_01158_gb300 import minimize
    row = [r for r in read_golden("benchmark6_lshape.txt") if int(r["level"]) == level][0]
    coords, elems, bnd = mg.lshape_tri(level)
    nn = coords.shape[0]
    w = mg.Workload(f"lshape{level}", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE_LP,
                    p=3.0, f=np.full(nn, -10.0), v=np.zeros(nn))
    gm = fem.FEMesh.from_workload(w)
    res = minimize.newton_cg(minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm),
                             torch.zeros(nn, dtype=torch.float64, device="cuda"), gtol=1e-10,
                             cg=minimize.mesh_cg(gm))
    assert res.converged
    assert abs(res.J - row["J_min"]) <= 5e-5, (res.J, row["J_min"])


def test_gpu_nested_newton_to_level7():
    """Nested iteration on the FP64 kernels and the device CG: levels 1..7, each started from
    the previous minimiser, every level's printed J(u) to its 4 decimals, few Newton steps per
    level."""
    fem = _fem()
    from paper_2109_01158_gb300 import minimize
    table = {int(r["level"]): r["J_min"] for r in read_golden("benchmark6_lshape.txt")}
    levels = []
    for L in range(1, 8):
        coords, elems, bnd = mg.lshape_tri(L)
        nn = coords.shape[0]
        w = mg.Workload(f"lshape{L}", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE_LP,
                        p=3.0, f=np.full(nn, -10.0), v=np.zeros(nn))
        gm = fem.FEMesh.from_workload(w)
        levels.append((minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm), minimize.mesh_cg(gm), coords, elems))
    n1 = mg.lshape_tri(1)[0].shape[0]
    res = minimize.nested_newton(levels, torch.zeros(n1, dtype=torch.float64, device="cuda"), gtol=1e-10)
    for L, r in zip(range(1, 8), res):
        assert r.converged and abs(r.J - table[L]) <= 5e-5, (L, r.J)
        if L > 1:
            assert r.iters <= 12, (L, r.iters)
