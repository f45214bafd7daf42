"""L-BFGS minimisation (the minimiser that replaces the paper's trust region).

CPU tests drive the minimiser with the oracle; GPU tests drive it with the kernels (FP64,
double-float, FP32, exact and central-difference gradients, and several instances in lockstep
through one batched launch per line-search round)."""
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
from paper_2109_01158_gb300.minimize import lbfgs, lbfgs_batched, newton_cg, torsion_continuation  # noqa: E402
from conftest import read_golden  # noqa: E402


def _oracle_ev(om):
    def ev(v):
        vv = v.cpu().numpy()
        J, _ = om.energy(vv)
        g, _ = om.gradient_exact(vv)
        return J, torch.from_numpy(g).to(v.device)
    return ev


def _lshape(level, p=3.0):
    coords, elems, bnd = mg.lshape_tri(level)
    nn = coords.shape[0]
    return mg.Workload(f"lshape{level}", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE,
                       p=p, f=np.full(nn, -10.0), v=np.zeros(nn))


def test_p2_minimiser_solves_the_five_point_system():
    """p = 2: the minimiser of v.Kv/2 - b.v solves K u = b; on the right-triangle grid K is the
    5-point Laplacian, solved here by a sparse direct solver (textbook reference)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n = 16
    w = mg.plaplace_square(n, p=2.0)
    om = oracle.OracleMesh(w)
    res = lbfgs(_oracle_ev(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-12)
    assert res.converged
    m = n - 1
    T = sp.diags([-1.0, 4.0, -1.0], [-1, 0, 1], shape=(m, m))
    K = sp.kron(sp.eye(m), T) + sp.kron(sp.diags([-1.0, -1.0], [-1, 1], shape=(m, m)), sp.eye(m))
    inner = (w.dirichlet == 0)
    u = spl.spsolve(K.tocsc(), om.b[inner])
    np.testing.assert_allclose(res.v.numpy()[inner], u, rtol=0, atol=1e-9 * np.abs(u).max())
    assert abs(res.J - (-0.5 * om.b[inner] @ u)) < 1e-10 * abs(res.J)


@pytest.mark.parametrize("p", [1.5, 3.0])
def test_plaplace_minimum_satisfies_euler_identity(p):
    """At the minimiser grad J_grad = b on free dofs, and J_grad is p-homogeneous, so
    b.u = p J_grad(u) and J(u) = (1/p - 1) b.u (the discrete Euler identity)."""
    w = _lshape(2, p)
    om = oracle.OracleMesh(w)
    res = lbfgs(_oracle_ev(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-11)
    assert res.converged and res.J < 0
    bu = float(om.b @ res.v.numpy())
    assert abs(res.J - (1.0 / p - 1.0) * bu) <= 1e-8 * abs(res.J)


def test_lbfgs_rejects_inverted_trial_points():
    """A first step that folds elements gets J = +Inf and is halved until it does not."""
    w = mg.neohooke_cube3d(3)
    w.f = np.tile([0.0, 0.0, -5e3], w.nn)
    w.v = w.coords.ravel().copy()
    om = oracle.OracleMesh(w)
    res = lbfgs(_oracle_ev(om), torch.from_numpy(w.v), gtol=1e-6, relative=True, max_iter=400)
    assert res.converged and math.isfinite(res.J)
    assert oracle.OracleMesh(w).energy(res.v.numpy())[1] == oracle.OK


def _oracle_hvp(om):
    def hvp(v, x):
        H, _ = om.hessian_vector(v.cpu().numpy(), x.cpu().numpy())
        return torch.from_numpy(H).to(v.device)
    return hvp


def test_newton_cg_p2_converges_in_one_step():
    """p = 2 is a quadratic: the first Newton step (CG to 1e-12) lands on the solution of
    the five-point system, the same minimiser as L-BFGS."""
    w = mg.plaplace_square(16, p=2.0)
    om = oracle.OracleMesh(w)
    res = newton_cg(_oracle_ev(om), _oracle_hvp(om), torch.zeros(w.nn, dtype=torch.float64),
                    gtol=1e-11, eta_max=1e-12)
    ref = lbfgs(_oracle_ev(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-12)
    assert res.converged and res.iters <= 3
    np.testing.assert_allclose(res.v.numpy(), ref.v.numpy(), atol=1e-9 * np.abs(ref.v.numpy()).max())


@pytest.mark.parametrize("p", [3.0, 4.5])
def test_newton_cg_lshape_matches_lbfgs(p):
    """The degenerate p-Laplacian (p > 2: the Hessian vanishes where grad v = 0, as at the
    start v = 0) on the L-shape: trust-region Newton-CG reaches the same minimum as L-BFGS,
    in far fewer iterations, and satisfies the Euler identity J = (1/p - 1) b.u."""
    w = _lshape(3, p)
    om = oracle.OracleMesh(w)
    res = newton_cg(_oracle_ev(om), _oracle_hvp(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-10)
    ref = lbfgs(_oracle_ev(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-10)
    assert res.converged and res.iters < ref.iters / 3
    assert abs(res.J - ref.J) <= 1e-11 * abs(ref.J)
    assert abs(res.J - (1.0 / p - 1.0) * float(om.b @ res.v.numpy())) <= 1e-8 * abs(res.J)


def _torsion_rows(level):
    return {int(r["t"]): r["J"] for r in read_golden("benchmark4_torsion.txt") if int(r["level"]) == level}


def _check_torsion(J, paper):
    """Our minimum is within 3e-4 of the printed one (which is rounded to 4 decimals and comes
    from a trust-region run stopped at its own tolerance).  Once the bar has buckled, the
    continuation passes near-singular Hessians and nearby stationary states: which of them a
    solver settles in depends on rounding (a change in the order of the patch sums moved the
    level-2 minimum at t = 24 from below the printed 116.3261 to 116.3363 above it), so the
    check is two-sided."""
    assert abs(J - paper) <= 3e-4 * abs(paper), (J, paper)


def test_torsion_continuation_first_steps_level1():
    """Benchmark 4 at level 1 (2133 free dofs), oracle-driven: the first three steps of the
    continuation reach the printed minimal energy of t = 3."""
    w = mg.twisted_bar(1)
    om = oracle.OracleMesh(w)
    coords = torch.from_numpy(w.coords)
    dirichlet = torch.from_numpy(w.dirichlet.astype(np.int64))
    last = None
    for t, r in torsion_continuation(_oracle_ev(om), _oracle_hvp(om), coords, dirichlet, T=24):
        assert r.converged
        last = r
        if t == 3:
            break
    _check_torsion(last.J, _torsion_rows(1)[3])


# ---------------------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------------------

def _gpu():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01158_gb300 import fem, minimize
    return fem, minimize


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_gpu_minimiser_matches_oracle_driven_minimiser(precision):
    fem, minimize = _gpu()
    w = _lshape(3)
    om = oracle.OracleMesh(w)
    ref = lbfgs(_oracle_ev(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-10)
    gm = fem.FEMesh.from_workload(w, precisions=(precision,))
    res = lbfgs(minimize.mesh_evaluator(gm), torch.zeros(w.nn, dtype=torch.float64, device="cuda"), gtol=1e-10)
    assert res.converged
    assert abs(res.J - ref.J) <= 1e-9 * abs(ref.J)
    np.testing.assert_allclose(res.v.cpu().numpy(), ref.v.numpy(), atol=1e-7)


@pytest.mark.gpu
def test_gpu_minimiser_fd_gradient_and_fp32_path():
    """Exact vs central-difference gradients and FP64 vs FP32 element arithmetic reach the
    same minimum to the accuracy each provides."""
    fem, minimize = _gpu()
    w = _lshape(3)
    gm = fem.FEMesh.from_workload(w, precisions=(fem.FE_F64, fem.FE_F32_COMP))
    z = torch.zeros(w.nn, dtype=torch.float64, device="cuda")
    ex = lbfgs(minimize.mesh_evaluator(gm, "exact"), z, gtol=1e-9)
    fd = lbfgs(minimize.mesh_evaluator(gm, "fd", eps=1e-5), z, gtol=1e-7)
    gm.set_precision(fem.FE_F32_COMP)
    f32 = lbfgs(minimize.mesh_evaluator(gm, "exact"), z, gtol=1e-5)
    assert ex.converged and fd.converged and f32.converged
    assert abs(fd.J - ex.J) <= 1e-8 * abs(ex.J)
    assert abs(f32.J - ex.J) <= 1e-6 * abs(ex.J)


@pytest.mark.gpu
def test_gpu_lockstep_instances_match_individual_runs():
    """Eight minimisations of different problems run in lockstep through the batched kernels
    reach the same minima as individual runs."""
    fem, minimize = _gpu()
    ws = []
    for k in range(8):
        if k % 2 == 0:
            w = _lshape(2 + (k % 4) // 2, p=(3.0, 1.5)[(k // 2) % 2])
        else:
            w = mg.neohooke_cube3d(4 + k // 2)
            w.f = np.tile([0.0, 0.0, -50.0], w.nn)
            w.v = w.coords.ravel().copy()
        ws.append(w)
    meshes = [fem.FEMesh.from_workload(w, precisions=(fem.FE_DF64,)) for w in ws]
    v0 = [torch.from_numpy(np.ascontiguousarray(w.v)).cuda() for w in ws]
    batch = fem.Batch(0)
    res = lbfgs_batched(minimize.batch_evaluator(batch, meshes), v0, gtol=1e-8, relative=True)
    for w, mesh, r, v in zip(ws, meshes, res, v0):
        single = lbfgs(minimize.mesh_evaluator(mesh), v, gtol=1e-8, relative=True)
        assert r.converged and single.converged
        assert abs(r.J - single.J) <= 1e-9 * max(abs(single.J), 1e-30) + 1e-14


@pytest.mark.gpu
def test_gpu_newton_cg_matches_oracle_driven_and_lbfgs():
    """Trust-region Newton-CG on the kernels' Hessian-vector products: the L-shape (p = 3,
    level 4) against the oracle-driven run, and the 3D gravity problem (16^3 x 6, displacement
    input) against L-BFGS on the kernels."""
    fem, minimize = _gpu()
    w = _lshape(4)
    om = oracle.OracleMesh(w)
    ref = newton_cg(_oracle_ev(om), _oracle_hvp(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-10)
    gm = fem.FEMesh.from_workload(w)
    z = torch.zeros(w.nn, dtype=torch.float64, device="cuda")
    res = newton_cg(minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm), z, gtol=1e-10)
    assert res.converged and ref.converged
    assert abs(res.J - ref.J) <= 1e-11 * abs(ref.J)
    w3 = mg.neohooke_cube3d(16)
    w3.f = np.tile([0.0, 0.0, -1e-2], w3.nn)
    g3 = fem.FEMesh.from_workload(w3)
    g3.set_input(fem.FE_INPUT_DISPLACEMENT)
    u0 = torch.zeros(w3.ndof, dtype=torch.float64, device="cuda")
    nt = newton_cg(minimize.mesh_evaluator(g3), minimize.mesh_hvp(g3), u0, gtol=1e-8, relative=True)
    lb = lbfgs(minimize.mesh_evaluator(g3), u0, gtol=1e-8, relative=True)
    assert nt.converged and lb.converged and nt.iters < lb.iters / 10
    assert abs(nt.J - lb.J) <= 1e-13 * abs(lb.J)


@pytest.mark.gpu
@pytest.mark.parametrize("level", [1, 2])
def test_gpu_torsion_continuation_reproduces_benchmark4(level):
    """Benchmark 4 on the FP64 kernels (energy, gradient, Hessian-vector products): all 24 steps
    of the continuation, every printed minimal energy of the table (t = 3, 6, ..., 24)."""
    fem, minimize = _gpu()
    w = mg.twisted_bar(level)
    gm = fem.FEMesh.from_workload(w)
    coords = torch.from_numpy(w.coords).cuda()
    dirichlet = torch.from_numpy(w.dirichlet.astype(np.int64)).cuda()
    rows = _torsion_rows(level)
    for t, r in torsion_continuation(minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm), coords, dirichlet,
                                     cg=minimize.mesh_cg(gm)):
        assert r.converged, (t, r.iters)
        if t in rows:
            _check_torsion(r.J, rows[t])


def test_lbfgs_batched_follows_each_instance_alone():
    """Jobs driven together take exactly the iterates of each job driven alone (CPU oracle)."""
    oms = []
    for k, p in enumerate((2.0, 3.0, 4.5)):
        w = mg.plaplace_square(8, p=p, f=-10.0 * (1 + k))
        w.v = np.zeros(w.nn)
        oms.append((w, oracle.OracleMesh(w)))

    def batch_eval(trials):
        return [_oracle_ev(oms[k][1])(v) for k, v in trials]
    res = lbfgs_batched(batch_eval, [torch.zeros(w.nn, dtype=torch.float64) for w, _ in oms], gtol=1e-9)
    for (w, om), r in zip(oms, res):
        single = lbfgs(_oracle_ev(om), torch.zeros(w.nn, dtype=torch.float64), gtol=1e-9)
        assert r.converged and single.converged
        assert r.J == single.J and r.iters == single.iters and r.evals == single.evals
        assert torch.equal(r.v, single.v)
