"""Hessian-vector products on the GPU (fe_hessian_vector, FP64) against the oracle's, which
the CPU tests pin to the 5-point Laplacian, symmetry, central differences of the gradient,
linear elasticity at F = I and decimal second derivatives."""
import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_grad

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


@pytest.mark.parametrize("seed,dim,model,p,n", [
    (71, 2, mg.MODEL_PLAPLACE, 3.0, (13, 11)), (72, 2, mg.MODEL_PLAPLACE, 1.5, (9, 8)),
    (73, 3, mg.MODEL_PLAPLACE, 4.5, (5, 4, 6)), (74, 2, mg.MODEL_PLAPLACE, 2.0, (7, 9)),
    (75, 2, mg.MODEL_NEOHOOKE, 0, (17, 13)), (76, 3, mg.MODEL_NEOHOOKE, 0, (6, 5, 7)),
    (77, 3, mg.MODEL_NEOHOOKE, 0, (1, 1, 1)),
])
@pytest.mark.parametrize("order", [0, 1])
def test_hessian_vector_matches_oracle(seed, dim, model, p, n, order):
    fem = _fem()
    w = mg.random_small(seed, dim, model, *n, p=p or 3.0)
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w, order=order)
    x = mg.uniform(seed + 1, np.arange(w.ndof), -1.0, 1.0)
    ref, st = om.hessian_vector(w.v, x)
    assert st == oracle.OK
    Hx = gm.hessian_vector(_dev(w.v), _dev(x)).cpu().numpy()
    assert gm.sync_status() == fem.FE_OK
    check_grad(Hx, ref)
    assert np.all(Hx[w.dirichlet == 1] == 0.0)


def test_hessian_vector_with_displacement_input():
    fem = _fem()
    w = mg.random_small(78, 3, mg.MODEL_NEOHOOKE, 5, 4, 4)
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w)
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    x = mg.uniform(79, np.arange(w.ndof), -1.0, 1.0)
    Hx = gm.hessian_vector(_dev(w.v - w.coords.ravel()), _dev(x)).cpu().numpy()
    check_grad(Hx, om.hessian_vector(w.v, x)[0])


def test_hessian_vector_c3_full():
    """3D Neo-Hookean 128^3 x 6 (12,582,912 tets): every dof against the oracle."""
    fem = _fem()
    w = mg.neohooke_cube3d(128)
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w)
    x = mg.uniform(80, np.arange(w.ndof), -1.0, 1.0)
    Hx = gm.hessian_vector(_dev(w.v), _dev(x)).cpu().numpy()
    check_grad(Hx, om.hessian_vector(w.v, x)[0])


@pytest.mark.parametrize("dim,model", [(2, mg.MODEL_NEOHOOKE), (3, mg.MODEL_NEOHOOKE), (2, mg.MODEL_PLAPLACE)])
def test_hessian_vector_symmetric_and_central_differences(dim, model):
    """u.Hw = w.Hu, and Hw agrees with central differences of the GPU gradient to O(h^2)."""
    fem = _fem()
    w = mg.random_small(81 + dim, dim, model, *((21, 17) if dim == 2 else (7, 6, 5)))
    gm = fem.FEMesh.from_workload(w)
    free = w.dirichlet == 0
    a = mg.uniform(83, np.arange(w.ndof), -1.0, 1.0) * free
    b = mg.uniform(84, np.arange(w.ndof), -1.0, 1.0) * free
    v = _dev(w.v)
    Ha = gm.hessian_vector(v, _dev(a)).cpu().numpy()
    Hb = gm.hessian_vector(v, _dev(b)).cpu().numpy()
    assert abs(b @ Ha - a @ Hb) <= 1e-12 * (np.abs(b) @ np.abs(Ha))
    h = 1e-4 / 7 if model == mg.MODEL_NEOHOOKE else 1e-4
    gp = gm.gradient_exact(_dev(w.v + h * a)).cpu().numpy()
    gn = gm.gradient_exact(_dev(w.v - h * a)).cpu().numpy()
    check_grad((gp - gn) / (2 * h), Ha, rtol=1e-6)
