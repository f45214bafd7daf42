"""The device-resident Steihaug CG (fe_cg_steihaug) against the same algorithm written with
torch vector operations over the library's Hessian-vector product: the same stopping reason,
the same number of products and the same step up to rounding, in each of its exits (residual
tolerance, trust-region boundary, non-positive curvature, iteration limit); bitwise
reproducible; and trust-region Newton-CG driven by it reaching the oracle's minimum."""
import numpy as np
import pytest

import oracle
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


def _lshape(level, v_seed=None):
    coords, elems, bnd = mg.lshape_tri(level)
    nn = coords.shape[0]
    v = np.zeros(nn) if v_seed is None else mg.uniform(v_seed, np.arange(nn), -0.5, 0.5) * (~bnd)
    return mg.Workload(f"lshape{level}", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE_LP,
                       p=3.0, f=np.full(nn, -10.0), v=v)


def _cases():
    """(name, workload): a deformed 3D Neo-Hookean block, a 2D Neo-Hookean plate and the
    componentwise p-Laplacian on the L-shape at a random point."""
    return [("nh3d", mg.random_small(61, 3, mg.MODEL_NEOHOOKE, 7, 6, 5)),
            ("nh2d", mg.random_small(62, 2, mg.MODEL_NEOHOOKE, 23, 19)),
            ("lp2d", _lshape(3, v_seed=63))]


def _reference(gm, v, g, radius, tol, max_cg, history=None):
    from paper_2109_01158_gb300.minimize import _cg_steihaug
    cnt = [0]

    def hv(w):
        cnt[0] += 1
        return gm.hessian_vector(v, w)
    z, Hz, k, bnd = _cg_steihaug(g, hv, radius, tol, max_cg, history)
    assert k == cnt[0]
    return z, Hz, k, bnd


def _separated_tol(gm, v, g, tol0):
    """A residual tolerance near tol0 that no step of the reference run meets by a hair: the
    geometric mean of the first residual norm <= tol0 and the smallest norm before it.  The
    device CG sums its dot products in another order than torch; a tolerance within rounding
    of a residual norm would let the two stop one step apart for that reason alone."""
    hist = []
    _, _, k, _ = _reference(gm, v, g, 1e30, tol0, 10000, hist)
    if k < 2:
        return tol0, k
    before = min(hist[:k - 1])
    assert before > 1.001 * hist[k - 1], (before, hist[k - 1])
    return (before * hist[k - 1]) ** 0.5, k


def _close(a, b, rel):
    scale = float(b.abs().max()) or 1.0
    assert float((a - b).abs().max()) <= rel * scale, (float((a - b).abs().max()), scale)


@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("regime", ["interior", "boundary", "limit"])
def test_device_cg_matches_torch_cg(case, regime):
    fem = _fem()
    name, w = _cases()[case]
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    _, g = gm.energy_gradient(v)
    gn = float(g.norm())
    tol0, _ = _separated_tol(gm, v, g, 1e-8 * gn)
    z_full, _, k_full, _ = _reference(gm, v, g, 1e30, tol0, 10000)
    radius, tol, max_cg = {"interior": (1e30, tol0, 10000),
                           "boundary": (0.3 * float(z_full.norm()), tol0, 10000),
                           "limit": (1e30, tol0, max(1, k_full // 3))}[regime]
    zr, Hzr, kr, br = _reference(gm, v, g, radius, tol, max_cg)
    z, Hz, k, b = gm.cg_steihaug(v, g, radius, tol, max_cg)
    assert (k, b) == (kr, br), (name, k, kr, b, br)
    assert b == (regime == "boundary")
    if regime == "limit":
        assert k == max_cg
    # a boundary step is pinned by the radius; a converged z or one at the iteration limit
    # comes after ~100 steps, over which the rounding differences of the two dot-product
    # orders grow (finite-precision CG loses orthogonality), so those get a wider bound
    rel = 1e-9 if regime == "boundary" else 1e-6
    _close(z, zr, rel)
    _close(Hz, Hzr, rel)
    if b:
        assert abs(float(z.norm()) - radius) <= 1e-12 * radius
    # the model decrease is the one the quadratic predicts from z and Hz
    assert float(torch.dot(g, z) + 0.5 * torch.dot(z, Hz)) < 0.0
    # bitwise reproducible
    z2, Hz2, k2, b2 = gm.cg_steihaug(v, g, radius, tol, max_cg)
    assert (k2, b2) == (k, b) and torch.equal(z2, z) and torch.equal(Hz2, Hz)


def test_device_cg_nonpositive_curvature_and_trivial_exits():
    """At v = 0 the p = 3 componentwise Hessian vanishes: the first direction has d.Hd = 0 and
    the step is -radius g / ||g||.  A gradient already below tol, or max_cg = 0, gives z = 0."""
    fem = _fem()
    w = _lshape(2)
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    _, g = gm.energy_gradient(v)
    z, Hz, k, b = gm.cg_steihaug(v, g, 0.25, 1e-12, 100)
    assert (k, b) == (1, True)
    _close(z, -0.25 * g / g.norm(), 1e-14)
    assert float(Hz.abs().max()) == 0.0
    for tol, max_cg in ((2.0 * float(g.norm()), 100), (0.0, 0)):
        z, Hz, k, b = gm.cg_steihaug(v, g, 1.0, tol, max_cg)
        assert (k, b) == (0, False) and float(z.abs().max()) == 0.0 and float(Hz.abs().max()) == 0.0


def test_device_cg_argument_errors():
    fem = _fem()
    w = _lshape(1)
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    _, g = gm.energy_gradient(v)
    for radius, tol, max_cg in ((0.0, 1e-8, 10), (float("inf"), 1e-8, 10), (1.0, -1.0, 10), (1.0, 1e-8, -1)):
        with pytest.raises(fem.FEError):
            gm.cg_steihaug(v, g, radius, tol, max_cg)


@pytest.mark.parametrize("level", [3, 4])
def test_newton_with_device_cg_reaches_the_oracle_minimum(level):
    fem = _fem()
    from paper_2109_01158_gb300 import minimize
    w = _lshape(level)
    om = oracle.OracleMesh(w)

    def ev(x):
        J, _ = om.energy(x.numpy())
        g, _ = om.gradient_exact(x.numpy())
        return J, torch.from_numpy(g)

    def hvp(x, y):
        return torch.from_numpy(om.hessian_vector(x.numpy(), y.numpy())[0])
    ref = minimize.newton_cg(ev, hvp, torch.zeros(w.nn, dtype=torch.float64), gtol=1e-10)
    gm = fem.FEMesh.from_workload(w)
    res = minimize.newton_cg(minimize.mesh_evaluator(gm), minimize.mesh_hvp(gm),
                             torch.zeros(w.nn, dtype=torch.float64, device="cuda"), gtol=1e-10,
                             cg=minimize.mesh_cg(gm))
    assert ref.converged and res.converged
    assert abs(res.J - ref.J) <= 1e-11 * abs(ref.J)


@pytest.mark.parametrize("case", range(3))
def test_cached_products_equal_fe_hessian_vector(case):
    """Inside the device CG the v-dependent terms of the Hessian are computed once per solve;
    one CG step from z = 0 returns Hz = a H(-g), which must agree with fe_hessian_vector to
    rounding."""
    fem = _fem()
    name, w = _cases()[case]
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    _, g = gm.energy_gradient(v)
    z, Hz, k, b = gm.cg_steihaug(v, g, 1e30, 0.0, 1)
    assert (k, b) == (1, False)
    i = int((-g).abs().argmax())
    a = float(z[i] / (-g[i]))
    ref = a * gm.hessian_vector(v, -g)
    assert float((Hz - ref).abs().max()) <= 1e-14 * float(ref.abs().max()), name


def test_device_cg_on_a_mesh_without_free_dofs():
    """Every dof fixed: the gradient is 0, so the solve stops before any product."""
    fem = _fem()
    w = _lshape(1)
    w.dirichlet[:] = 1
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    _, g = gm.energy_gradient(v)
    assert float(g.abs().max()) == 0.0
    z, Hz, k, b = gm.cg_steihaug(v, g, 1.0, 0.0, 10)
    assert (k, b) == (0, False) and float(z.abs().max()) == 0.0
