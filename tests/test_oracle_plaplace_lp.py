"""Pins of the componentwise p-Laplacian (model 2: W = (1/p) sum_m |dv/dx_m|^p, eq. pLaplacian
read with the l^p norm of the gradient) in the oracle, and the minimal energies of the
Benchmark 6 table, which this reading reproduces to the printed digits."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2109_01158_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
from paper_2109_01158_gb300.minimize import newton_cg  # noqa: E402


def _lp(w):
    w.model = mg.MODEL_PLAPLACE_LP
    return w


def _lshape_lp(level, p=3.0):
    coords, elems, bnd = mg.lshape_tri(level)
    nn = coords.shape[0]
    return mg.Workload(f"lshape{level}", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE_LP,
                       p=p, f=np.full(nn, -10.0), v=np.zeros(nn))


@pytest.mark.parametrize("p", [1.5, 3.0, 4.5])
def test_linear_field_closed_form(p):
    """v = a.x on the unit square: J_grad = |Omega| (|a_1|^p + |a_2|^p) / p, and the gradient
    vanishes at the interior nodes (a linear field is stationary for any density of grad v)."""
    w = _lp(mg.plaplace_square(8, p=p))
    w.f = None
    a = np.array([0.7, -1.3])
    w.v = w.coords @ a
    om = oracle.OracleMesh(w)
    J, st = om.energy(w.v)
    assert st == oracle.OK
    ref = (abs(a[0]) ** p + abs(a[1]) ** p) / p
    assert abs(J - ref) <= 1e-13 * ref
    g, _ = om.gradient_exact(w.v)
    bnd = mg.plaplace_square(8, p=p).dirichlet == 1
    assert np.abs(g[~bnd]).max() <= 1e-12


@pytest.mark.parametrize("p", [1.5, 3.0])
def test_euler_identity(p):
    """W is positively homogeneous of degree p: sum_n v_n dJ_grad/dv_n = p J_grad."""
    w = _lp(mg.random_small(31, 2, mg.MODEL_PLAPLACE, 9, 7, p=p))
    w.f = None
    w.dirichlet[:] = 0
    om = oracle.OracleMesh(w)
    J, _ = om.energy(w.v)
    g, _ = om.gradient_exact(w.v)
    assert abs(float(w.v @ g) - p * J) <= 1e-12 * abs(p * J)


def test_p2_equals_the_euclidean_model():
    w = mg.random_small(32, 2, mg.MODEL_PLAPLACE, 8, 6, p=2.0)
    e = oracle.OracleMesh(w)
    l2 = oracle.OracleMesh(_lp(mg.random_small(32, 2, mg.MODEL_PLAPLACE, 8, 6, p=2.0)))
    assert abs(e.energy(w.v)[0] - l2.energy(w.v)[0]) <= 1e-14 * abs(e.energy(w.v)[0])
    np.testing.assert_allclose(l2.gradient_exact(w.v)[0], e.gradient_exact(w.v)[0], rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_and_hessian_central_differences(dim):
    """Exact gradient vs central differences of J, and the Hessian-vector product vs central
    differences of the gradient (errors falling by 4 as h halves; p = 4.5, where W is not a
    piecewise polynomial that central differences would reproduce exactly), and symmetry of
    the Hessian."""
    w = _lp(mg.random_small(33 + dim, dim, mg.MODEL_PLAPLACE, *((7, 6) if dim == 2 else (3, 4, 3)), p=4.5))
    om = oracle.OracleMesh(w)
    free = w.dirichlet == 0
    x = mg.uniform(35, np.arange(w.ndof), -1.0, 1.0) * free
    g, _ = om.gradient_exact(w.v)
    Hx, _ = om.hessian_vector(w.v, x)
    errs_g, errs_h = [], []
    for h in (4e-3, 2e-3, 1e-3):
        Jp, _ = om.energy(w.v + h * x)
        Jm, _ = om.energy(w.v - h * x)
        errs_g.append(abs((Jp - Jm) / (2 * h) - float(g @ x)))
        gp, _ = om.gradient_exact(w.v + h * x)
        gm, _ = om.gradient_exact(w.v - h * x)
        errs_h.append(np.abs((gp - gm) / (2 * h) - Hx).max())
    for errs in (errs_g, errs_h):
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    y = mg.uniform(36, np.arange(w.ndof), -1.0, 1.0) * free
    Hy, _ = om.hessian_vector(w.v, y)
    assert abs(float(y @ Hx) - float(x @ Hy)) <= 1e-12 * (np.abs(y) @ np.abs(Hx))


def _newton_oracle(om, n):
    def ev(v):
        J, _ = om.energy(v.numpy())
        g, _ = om.gradient_exact(v.numpy())
        return J, torch.from_numpy(g)

    def hvp(v, x):
        H, _ = om.hessian_vector(v.numpy(), x.numpy())
        return torch.from_numpy(H)
    return newton_cg(ev, hvp, torch.zeros(n, dtype=torch.float64), gtol=1e-10)


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_benchmark6_minimal_energies(level):
    """The L-shape of Benchmark 6 (p = 3, f = -10, zero Dirichlet data): the minimum of the
    componentwise reading equals the printed J(u) of the table to its 4 decimals."""
    row = [r for r in read_golden("benchmark6_lshape.txt") if int(r["level"]) == level][0]
    w = _lshape_lp(level)
    assert int((w.dirichlet == 0).sum()) == int(row["free_dofs"])
    res = _newton_oracle(oracle.OracleMesh(w), w.nn)
    assert res.converged
    assert abs(res.J - row["J_min"]) <= 5e-5, (res.J, row["J_min"])
