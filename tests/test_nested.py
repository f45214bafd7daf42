"""Nested iteration (minimize.prolongation_pairs, prolong, nested_newton).  On uniformly
refined meshes the coarse P1 space is a subspace of the fine one, so the prolonged function
is the same function: its energy on the fine mesh equals its energy on the coarse mesh to
rounding (the load term too, since b = M f integrates a P1 load exactly).  Nested Newton
reaches the Benchmark 6 minima with a few iterations per level."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2109_01158_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
from paper_2109_01158_gb300 import minimize as M  # noqa: E402


def _lshape(level, v=None):
    c, e, b = mg.lshape_tri(level)
    return mg.Workload(f"lshape{level}", 2, 1, c, e, b.astype(np.uint8), mg.MODEL_PLAPLACE_LP, p=3.0,
                       f=np.full(c.shape[0], -10.0), v=np.zeros(c.shape[0]) if v is None else v)


def _box(n, v=None):
    X, E = mg.box_tet(n, n, n)
    dmask = np.repeat(np.abs(X[:, 0]) < 1e-12, 3).astype(np.uint8)
    C1, D1 = mg.lame_c1_d1(1e4, 0.3)
    return X, E, mg.Workload(f"box{n}", 3, 3, X, E, dmask, mg.MODEL_NEOHOOKE, C1=C1, D1=D1,
                             f=np.tile([0.0, 0.0, -1.0], X.shape[0]), v=v)


def test_prolongation_preserves_the_energy_2d():
    c, e, b = mg.lshape_tri(2)
    v = mg.uniform(5, np.arange(c.shape[0]), -1.0, 1.0) * (~b)
    cf, _, bf = mg.lshape_tri(3)
    pairs = M.prolongation_pairs(c, e, cf)
    vf = M.prolong(torch.from_numpy(v), pairs).numpy()
    assert np.all(vf[bf] == 0.0)
    Jc = oracle.OracleMesh(_lshape(2, v)).energy(v)[0]
    Jf = oracle.OracleMesh(_lshape(3, vf)).energy(vf)[0]
    assert abs(Jf - Jc) <= 1e-14 * abs(Jc)
    # a linear field is reproduced exactly at every fine node
    a = np.array([0.3, -0.7])
    np.testing.assert_allclose(M.prolong(torch.from_numpy(c @ a), pairs).numpy(), cf @ a, rtol=0, atol=1e-15)


def test_prolongation_preserves_the_energy_3d_neohooke():
    X, E, _ = _box(2)
    v = X.ravel() + mg.uniform(7, np.arange(X.size), -0.05, 0.05)
    Xf, _, _ = _box(4)
    vf = M.prolong(torch.from_numpy(v), M.prolongation_pairs(X, E, Xf), d=3).numpy()
    J = oracle.OracleMesh(_box(2, v)[2]).energy(v)[0]
    Jf = oracle.OracleMesh(_box(4, vf)[2]).energy(vf)[0]
    assert abs(Jf - J) <= 1e-14 * abs(J)


def test_prolongation_rejects_meshes_that_are_not_nested():
    c, e = mg.rect_tri(4, 4)
    cf, _ = mg.rect_tri(6, 6)
    with pytest.raises(ValueError):
        M.prolongation_pairs(c, e, cf)


def test_nested_newton_reaches_the_benchmark6_minima():
    table = {int(r["level"]): r["J_min"] for r in read_golden("benchmark6_lshape.txt")}
    levels = []
    for L in range(1, 5):
        w = _lshape(L)
        om = oracle.OracleMesh(w)

        def ev(x, om=om):
            J, _ = om.energy(x.numpy())
            g, _ = om.gradient_exact(x.numpy())
            return J, torch.from_numpy(g)

        def hvp(x, y, om=om):
            return torch.from_numpy(om.hessian_vector(x.numpy(), y.numpy())[0])
        levels.append((ev, hvp, None, w.coords, w.elems))
    res = M.nested_newton(levels, torch.zeros(_lshape(1).nn, dtype=torch.float64), gtol=1e-10)
    for L, r in zip(range(1, 5), res):
        assert r.converged and abs(r.J - table[L]) <= 5e-5, (L, r.J)
        if L > 1:
            assert r.iters <= 10, (L, r.iters)
