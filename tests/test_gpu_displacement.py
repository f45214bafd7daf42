"""Displacement input (fe_set_input(FE_INPUT_DISPLACEMENT)): the evaluation calls take
u = v - X instead of the deformation v (Sec. 3 names v the unknown; F = grad v = I + grad u).

The results are those of the deformation v = X + u against the oracle at the usual
tolerances, in every precision and through the central-difference and batched calls; and
displacements far below the spacing of doubles near X keep their relative precision."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["f64", "f32", "df64"])
@pytest.mark.parametrize("seed,dim,n", [(21, 2, (9, 8)), (22, 3, (5, 4, 4))])
def test_displacement_input_matches_oracle(precision, seed, dim, n):
    fem = _fem()
    w = mg.random_small(seed, dim, mg.MODEL_NEOHOOKE, *n)
    u = w.v - w.coords.ravel()
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w, precisions=(precision, fem.FE_F64) if precision else (0,))
    gm.set_precision(precision)
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    J, g = gm.energy_gradient(_dev(u))
    Jref, _ = om.energy(w.v)
    gref, _ = om.gradient_exact(w.v)
    if precision == fem.FE_F32_COMP:           # the FP32 path's stated error bars
        check_energy(J.item(), Jref, energy_scale(om, w.v), rtol=2e-6)
        check_grad(g.cpu().numpy(), gref, rtol=2e-5)
    else:
        check_energy(J.item(), Jref, energy_scale(om, w.v))
        check_grad(g.cpu().numpy(), gref)
    # the central differences (FP64) read the same displacement
    gfd = gm.gradient_fd(_dev(u), 1e-6).cpu().numpy()
    check_grad(gfd, om.gradient_fd(w.v, 1e-6)[0], extra_abs=fd_extra(om, w.v, 1e-6))


def test_displacement_input_in_a_batch():
    """A batched request on a displacement-input mesh equals the oracle at v = X + u."""
    fem = _fem()
    w = mg.random_small(23, 3, mg.MODEL_NEOHOOKE, 4, 5, 3)
    u = w.v - w.coords.ravel()
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w, precisions=(fem.FE_DF64,))
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    dev = torch.device("cuda", 0)
    wb = fem.Batch.work_bytes(gm)
    buf = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    J = torch.empty((), dtype=torch.float64, device=dev)
    g = torch.empty(gm.ndof, dtype=torch.float64, device=dev)
    batch = fem.Batch(0)
    batch.run([(gm, _dev(u), J, g, buf[off: off + wb])])
    assert batch.sync_status() == fem.FE_OK
    check_energy(J.item(), om.energy(w.v)[0], energy_scale(om, w.v))
    check_grad(g.cpu().numpy(), om.gradient_exact(w.v)[0])


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_small_displacements_keep_their_precision(precision):
    """u ~ 1e-10 with no load: the gradient is linear in u up to O(|grad u|) ~ 1e-9 relative,
    so ||g(2u) - 2 g(u)|| <= 1e-8 ||g(u)|| with displacement input.  Passed as deformations,
    X + u rounds u to the spacing of doubles near X (about 1e-16, i.e. 1e-6 of u), and the
    same check is off by orders of magnitude."""
    fem = _fem()
    w = mg.neohooke_cube3d(6)
    w.f = None
    u = mg.uniform(31, np.arange(w.ndof), -1e-10, 1e-10) * (w.dirichlet == 0)
    gm = fem.FEMesh.from_workload(w, precisions=(precision,))

    def lin_err():
        g1 = gm.gradient_exact(_dev(u) if gm.input else _dev(w.coords.ravel() + u)).cpu().numpy()
        g2 = gm.gradient_exact(_dev(2 * u) if gm.input else _dev(w.coords.ravel() + 2 * u)).cpu().numpy()
        return np.abs(g2 - 2 * g1).max() / np.abs(g1).max()

    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    e_disp = lin_err()
    gm.set_input(fem.FE_INPUT_DEFORMATION)
    e_def = lin_err()
    assert e_disp <= 1e-8, e_disp
    assert e_def > 100 * e_disp, (e_def, e_disp)


def test_minimiser_in_displacement_form_goes_below_the_deformation_floor():
    """3D Neo-Hookean 16^3 x 6 under gravity (0, 0, -1e-2) from u = 0: L-BFGS on the
    displacement reaches ||g||_inf <= 1e-9 ||g_0||_inf, and its minimum agrees with the
    minimiser run on deformations to the accuracy that run reaches."""
    fem = _fem()
    from paper_2109_01158_gb300.minimize import lbfgs, mesh_evaluator
    w = mg.neohooke_cube3d(16)
    w.f = np.tile([0.0, 0.0, -1e-2], w.nn)
    gm = fem.FEMesh.from_workload(w, precisions=(fem.FE_F64,))
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    r = lbfgs(mesh_evaluator(gm), torch.zeros(w.ndof, dtype=torch.float64, device="cuda"),
              gtol=1e-9, relative=True, max_iter=20000)
    assert r.converged, (r.iters, r.gnorm / r.history[0][1])
    gm.set_input(fem.FE_INPUT_DEFORMATION)
    rd = lbfgs(mesh_evaluator(gm), _dev(w.coords.ravel()), gtol=1e-6, relative=True, max_iter=20000)
    assert rd.converged
    assert abs(r.J - rd.J) <= 1e-12 * abs(rd.J)
    # the displacement minimiser is a minimiser of the deformation problem too
    g = gm.gradient_exact(_dev(w.coords.ravel()) + r.v).cpu().numpy()
    assert np.abs(g).max() <= 1e-6 * r.history[0][1]
