"""Pins of the oracle's Hessian-vector product Hw = d/dt grad J(v + t w) (the second
derivative of the energy of Sec. 1 along w, gathered like the exact gradient of Sec. 6.2).

Each pin checks it against something other than its own formula: the 5-point Laplacian for
p = 2, the symmetry of a Hessian, central differences of the (separately pinned) exact
gradient, the textbook linear-elasticity stiffness at F = I, and the second derivative of
W at a homogeneous deformation in 50-digit decimal arithmetic."""
import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg


def _rand(seed, n):
    return mg.uniform(seed, np.arange(n), -1.0, 1.0)


def test_hessian_p2_is_the_five_point_laplacian():
    """p = 2: J_grad = v.Kv/2, so Hw = Kw, which on the right-triangle grid is the 5-point
    stencil at the interior nodes, whatever v."""
    n = 12
    w = mg.plaplace_square(n, p=2.0)
    om = oracle.OracleMesh(w)
    x = _rand(7, w.nn) * (w.dirichlet == 0)
    Hx, st = om.hessian_vector(w.v, x)
    assert st == oracle.OK
    X = x.reshape(n + 1, n + 1)
    st5 = 4 * X[1:-1, 1:-1] - X[1:-1, 2:] - X[1:-1, :-2] - X[2:, 1:-1] - X[:-2, 1:-1]
    np.testing.assert_allclose(Hx.reshape(n + 1, n + 1)[1:-1, 1:-1], st5, rtol=0, atol=1e-13)
    assert np.all(Hx[w.dirichlet == 1] == 0.0)


@pytest.mark.parametrize("dim,model,p", [(2, mg.MODEL_PLAPLACE, 3.0), (3, mg.MODEL_PLAPLACE, 4.5),
                                         (2, mg.MODEL_NEOHOOKE, 0), (3, mg.MODEL_NEOHOOKE, 0)])
def test_hessian_is_symmetric(dim, model, p):
    w = mg.random_small(40 + dim, dim, model, *((6, 5) if dim == 2 else (3, 4, 3)), p=p or 3.0)
    om = oracle.OracleMesh(w)
    a, b = _rand(1, w.ndof), _rand(2, w.ndof)
    Ha, _ = om.hessian_vector(w.v, a)
    Hb, _ = om.hessian_vector(w.v, b)
    free = w.dirichlet == 0
    lhs, rhs = float(b[free] @ Ha[free]), float(a[free] @ Hb[free])
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(b[free]) @ np.abs(Ha[free]))
    # a Hessian of a convex density near F = I (Neo-Hookean) / of |grad v|^p is positive
    assert float(a[free] @ Ha[free]) > 0


@pytest.mark.parametrize("dim,model", [(2, mg.MODEL_PLAPLACE), (2, mg.MODEL_NEOHOOKE),
                                       (3, mg.MODEL_NEOHOOKE)])
def test_hessian_matches_central_differences_of_the_gradient(dim, model):
    """(g(v + h w) - g(v - h w)) / 2h = Hw + O(h^2): the error falls by 4 when h halves."""
    w = mg.random_small(50 + dim, dim, model, *((7, 6) if dim == 2 else (3, 3, 4)))
    om = oracle.OracleMesh(w)
    x = _rand(3, w.ndof) * (w.dirichlet == 0)
    scale = 1e-2 * (1.0 / 7 if model == mg.MODEL_NEOHOOKE else 1.0)
    Hx, _ = om.hessian_vector(w.v, x)
    errs = []
    for h in (4 * scale, 2 * scale, scale):
        gp, _ = om.gradient_exact(w.v + h * x)
        gm, _ = om.gradient_exact(w.v - h * x)
        errs.append(np.abs((gp - gm) / (2 * h) - Hx).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] <= 1e-3 * np.abs(Hx).max()


def _voigt_stiffness(om, mu, lam):
    """Textbook P1 linear-elasticity stiffness: K_T = |T| B^T C B with the engineering-strain
    matrix B of the shape gradients and the isotropic C (Lame constants mu, lambda)."""
    dim, k = om.dim, om.dim + 1
    nv = 3 if dim == 2 else 6
    if dim == 2:
        C = np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])
    else:
        C = np.zeros((6, 6))
        C[:3, :3] = lam
        C[np.arange(3), np.arange(3)] += 2 * mu
        C[np.arange(3, 6), np.arange(3, 6)] = mu
    K = np.zeros((om.nn * dim, om.nn * dim))
    dphi = om.dphi.reshape(om.ne, k, dim)
    for e in range(om.ne):
        B = np.zeros((nv, k * dim))
        for l in range(k):
            gx = dphi[e, l]
            if dim == 2:
                B[0, 2 * l], B[1, 2 * l + 1] = gx[0], gx[1]
                B[2, 2 * l], B[2, 2 * l + 1] = gx[1], gx[0]
            else:
                c = 3 * l
                B[0, c], B[1, c + 1], B[2, c + 2] = gx[0], gx[1], gx[2]
                B[3, c + 1], B[3, c + 2] = gx[2], gx[1]      # gamma_yz
                B[4, c], B[4, c + 2] = gx[2], gx[0]          # gamma_xz
                B[5, c], B[5, c + 1] = gx[1], gx[0]          # gamma_xy
        Ke = om.vol[e] * B.T @ C @ B
        idx = (dim * om.elems[e][:, None] + np.arange(dim)[None, :]).ravel()
        K[np.ix_(idx, idx)] += Ke
    return K


@pytest.mark.parametrize("dim", [2, 3])
def test_hessian_at_identity_is_linear_elasticity(dim):
    """At v = X (F = I) the Neo-Hookean density linearises to sigma = 2 mu eps + lambda tr(eps) I
    with mu = 2 C1 and lambda = 2 D1, so Hw = K w with the textbook stiffness K."""
    w = mg.random_small(60 + dim, dim, mg.MODEL_NEOHOOKE, *((4, 3) if dim == 2 else (2, 2, 2)))
    om = oracle.OracleMesh(w)
    K = _voigt_stiffness(om, 2 * w.C1, 2 * w.D1)
    x = _rand(4, w.ndof) * (w.dirichlet == 0)
    Hx, st = om.hessian_vector(w.coords.ravel(), x)
    assert st == oracle.OK
    free = w.dirichlet == 0
    ref = (K @ x)[free]
    np.testing.assert_allclose(Hx[free], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def _w_decimal(A, C1, D1, dim):
    from decimal import Decimal
    a = [[Decimal(x) for x in row] for row in A]
    if dim == 2:
        det = a[0][0] * a[1][1] - a[0][1] * a[1][0]
    else:
        det = (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
               + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
    I1 = sum(x * x for row in a for x in row)
    return Decimal(C1) * (I1 - dim - 2 * det.ln()) + Decimal(D1) * (det - 1) ** 2


@pytest.mark.parametrize("dim", [2, 3])
def test_hessian_quadratic_form_at_a_homogeneous_deformation(dim):
    """v = A X and w = dA X on an all-free unit square / cube: every element has F = A and
    dF = dA, so w.Hw = |Omega| d^2/dt^2 W(A + t dA) at t = 0, computed here by a second
    difference in 50-digit decimals (h = 1e-15, error ~h^2)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    w = mg.neohooke_cube3d(3) if dim == 3 else mg.neohooke_rect2d(4, 4)
    w.dirichlet[:] = 0
    om = oracle.OracleMesh(w)
    rng = np.random.default_rng(5)
    A = np.eye(dim) + 0.3 * rng.standard_normal((dim, dim))
    if np.linalg.det(A) < 0.3:
        A = np.eye(dim) + 0.1 * rng.standard_normal((dim, dim))
    dA = rng.standard_normal((dim, dim))
    X = w.coords
    v = (X @ A.T).ravel()
    x = (X @ dA.T).ravel()
    Hx, st = om.hessian_vector(v, x)
    assert st == oracle.OK
    area = float(om.vol.sum())
    h = Decimal("1e-15")
    Ad = [[Decimal(repr(float(t))) for t in row] for row in A]
    dAd = [[Decimal(repr(float(t))) for t in row] for row in dA]
    Wt = lambda s: _w_decimal([[Ad[i][j] + s * dAd[i][j] for j in range(dim)] for i in range(dim)],
                              repr(w.C1), repr(w.D1), dim)
    d2 = float((Wt(h) - 2 * Wt(Decimal(0)) + Wt(-h)) / (h * h))
    # the mesh coordinates are exact in binary, v = A X is rounded: allow for that
    assert abs(float(x @ Hx) - area * d2) <= 1e-10 * abs(area * d2)
