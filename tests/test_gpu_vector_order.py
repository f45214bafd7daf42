"""Dof vectors in the device numbering (fe_set_vector_order(FE_VECTORS_DEVICE)): on a mesh
renumbered along a Morton curve, every evaluation in device order is the caller-order one
permuted, bit for bit (the node preparation, the element kernels and the patch sums see the
same values in the same order); the conversions are exact inverses; a minimisation run in
device order reaches the same minimum."""
import numpy as np
import pytest

from paper_2109_01158_gb300 import meshgen as mg

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


@pytest.mark.parametrize("order", [1, 2], ids=["morton", "rcm"])
@pytest.mark.parametrize("dim,model", [(3, mg.MODEL_NEOHOOKE), (2, mg.MODEL_PLAPLACE)])
@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_device_order_is_the_permuted_caller_order(dim, model, precision, order):
    fem = _fem()
    w = mg.shuffle_nodes(mg.random_small(71 + dim, dim, model, *((6, 5, 4) if dim == 3 else (19, 17))))
    gm = fem.FEMesh.from_workload(w, order=order, precisions=(precision, fem.FE_F64))
    v = _dev(w.v)
    x = _dev(mg.uniform(5, np.arange(w.ndof), -1.0, 1.0))
    J, g = gm.energy_gradient(v)
    Hx = gm.hessian_vector(v, x)
    gm.set_precision(fem.FE_F64)
    gfd = gm.gradient_fd(v, 1e-6)
    gm.set_precision(precision)
    vd, xd = gm.to_device_order(v), gm.to_device_order(x)
    assert not torch.equal(vd, v)                       # the numbering really differs
    assert torch.equal(gm.from_device_order(vd), v)     # exact inverse
    # the device numbering is the host-side renumbering fe_node_order reports
    perm = torch.from_numpy(fem.node_order(w.coords, w.elems, order).astype(np.int64)).cuda()
    d = w.ndof // w.nn
    assert torch.equal(vd.view(-1, d), v.view(-1, d)[perm])
    gm.set_vector_order(fem.FE_VECTORS_DEVICE)
    Jd, gd = gm.energy_gradient(vd)
    assert float(Jd) == float(J)
    assert torch.equal(gm.from_device_order(gd), g)
    assert torch.equal(gm.from_device_order(gm.hessian_vector(vd, xd)), Hx)
    gm.set_precision(fem.FE_F64)
    assert torch.equal(gm.from_device_order(gm.gradient_fd(vd, 1e-6)), gfd)
    # a dof subset is given in the device numbering too: the caller's dof of device dof k is
    # entry k of the caller's index vector moved to the device numbering
    dofs = np.array([0, 7, w.ndof - 1, 3], dtype=np.int64)
    sub = gm.gradient_fd(vd, 1e-6, dofs)
    gm.set_vector_order(fem.FE_VECTORS_CALLER)
    caller_of = gm.to_device_order(torch.arange(w.ndof, dtype=torch.float64, device="cuda"))
    caller_dofs = caller_of[torch.from_numpy(dofs).cuda()].long().cpu().numpy()
    assert torch.equal(sub, gm.gradient_fd(v, 1e-6, caller_dofs))
    gm.set_precision(precision)
    J2, g2 = gm.energy_gradient(v)
    assert float(J2) == float(J) and torch.equal(g2, g)


def test_minimisation_in_device_order():
    fem = _fem()
    from paper_2109_01158_gb300 import minimize
    w = mg.shuffle_nodes(mg.neohooke_cube3d(10))
    w.f = np.tile([0.0, 0.0, -1e-2], w.nn)
    gm = fem.FEMesh.from_workload(w, order=fem.FE_ORDER_MORTON)
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    u0 = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    ref = minimize.newton_cg(minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm), u0, gtol=1e-8, relative=True,
                             cg=minimize.mesh_cg(gm))
    gm.set_vector_order(fem.FE_VECTORS_DEVICE)
    res = minimize.newton_cg(minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm), gm.to_device_order(u0),
                             gtol=1e-8, relative=True, cg=minimize.mesh_cg(gm))
    assert ref.converged and res.converged
    assert abs(res.J - ref.J) <= 1e-13 * abs(ref.J)
    u = gm.from_device_order(res.v)
    assert float((u - ref.v).abs().max()) <= 1e-9 * float(ref.v.abs().max())


def test_vector_order_arguments():
    fem = _fem()
    w = mg.random_small(75, 2, mg.MODEL_PLAPLACE, 6, 5)
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    with pytest.raises(fem.FEError):
        gm.set_vector_order(2)
    with pytest.raises(fem.FEError):
        gm.to_device_order(v, out=v)
    # without a renumbering the device numbering is the caller's
    assert torch.equal(gm.to_device_order(v), v)
