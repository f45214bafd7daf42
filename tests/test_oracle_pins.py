"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values printed in the
paper, closed forms, invariants, textbook special cases, derivatives taken a different
way, or brute force on tiny meshes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from conftest import read_golden


def _free_all(w):
    w.dirichlet = np.zeros_like(w.dirichlet)
    return w


# ---------------------------------------------------------------------------------
# Mesh precompute (Sec. 4.1): volumes and P1 shape-function gradients
# ---------------------------------------------------------------------------------

def _single(dim, pts):
    coords = np.array(pts, dtype=np.float64)
    elems = np.arange(dim + 1, dtype=np.int32)[None, :]
    d = 1
    w = mg.Workload("single", dim, d, coords, elems, np.zeros(dim + 1, np.uint8),
                    mg.MODEL_PLAPLACE, p=2.0, v=np.zeros(dim + 1))
    return oracle.OracleMesh(w)


def test_reference_triangle_and_tetrahedron():
    om = _single(2, [[0, 0], [1, 0], [0, 1]])
    np.testing.assert_array_equal(om.dphi.reshape(3, 2), [[-1, -1], [1, 0], [0, 1]])
    assert om.vol[0] == 0.5
    om = _single(3, [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    np.testing.assert_array_equal(om.dphi.reshape(4, 3),
                                  [[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    assert om.vol[0] == 1.0 / 6.0


@pytest.mark.parametrize("dim", [2, 3])
def test_shape_gradients_interpolate_vertices(dim):
    """phi_l(x_k) = delta_lk on every element: (x_k - x_0).grad(phi_l) = delta_lk - delta_l0,
    and |T| equals the simplex measure from the Cayley-Menger-free formula |det|/dim!."""
    w = mg.random_small(5, dim, mg.MODEL_NEOHOOKE, 4, 3, 3)
    om = oracle.OracleMesh(w)
    k = dim + 1
    X = om.coords[om.elems]                           # ne x k x dim
    G = om.dphi.reshape(om.ne, k, dim)
    lhs = np.einsum("ekm,elm->elk", X - X[:, :1, :], G)   # (x_k - x_0).grad phi_l
    target = np.eye(k)[None] - np.eye(k)[:, :1][None]
    np.testing.assert_allclose(lhs, np.broadcast_to(target, lhs.shape), atol=1e-12)
    E = (X[:, 1:, :] - X[:, :1, :])
    vol_ref = np.abs(np.linalg.det(E)) / math.factorial(dim)
    np.testing.assert_allclose(om.vol, vol_ref, rtol=1e-13)


@pytest.mark.parametrize("maker,area", [
    (lambda: mg.plaplace_square(8), 1.0),
    (lambda: mg.neohooke_rect2d(16, 8), 2.0),
    (lambda: mg.neohooke_cube3d(5), 1.0),
    (lambda: mg.twisted_bar(1), 0.4 * 0.01 * 0.01),
])
def test_volumes_sum_to_domain_measure(maker, area):
    om = oracle.OracleMesh(maker())
    assert abs(om.vol.sum() - area) <= 1e-13 * area


def test_lshape_area():
    coords, elems, bnd = mg.lshape_tri(2)
    w = mg.Workload("L", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE, p=3.0,
                    v=np.zeros(coords.shape[0]))
    om = oracle.OracleMesh(w)
    assert abs(om.vol.sum() - 3.0) < 1e-13


# ---------------------------------------------------------------------------------
# Linear term b = M f (eqs. mass2D, linearTerm2, linearTerm3)
# ---------------------------------------------------------------------------------

def test_mass_vector_integrates_products():
    """For f, w in V_h, (M f).w = int f w dx.  Unit square: f = 1 gives sum b = 1;
    f = x, w = x gives int x^2 = 1/3; f = x, w = y gives 1/4 (a lumped mass would fail
    the second and third)."""
    w = mg.plaplace_square(16)
    om = oracle.OracleMesh(w)
    x, y = om.coords[:, 0], om.coords[:, 1]
    om.set_load(np.ones(om.nn))
    assert abs(om.b.sum() - 1.0) < 1e-14
    om.set_load(x.copy())
    assert abs(om.b @ x - 1.0 / 3.0) < 1e-14
    assert abs(om.b @ y - 1.0 / 4.0) < 1e-14


def test_mass_vector_3d_vector_valued():
    w = mg.neohooke_cube3d(4)
    om = oracle.OracleMesh(w)
    f = np.tile([1.0, 2.0, -3.0], om.nn)
    om.set_load(f)
    np.testing.assert_allclose(om.b.reshape(-1, 3).sum(axis=0), [1.0, 2.0, -3.0], atol=1e-14)
    z = om.coords[:, 2]
    om.set_load(np.repeat(z, 3))                      # f^(j) = z for every component
    np.testing.assert_allclose(om.b.reshape(-1, 3).T @ z, [1 / 3] * 3, atol=1e-14)


# ---------------------------------------------------------------------------------
# Energy: values printed in the paper and closed forms
# ---------------------------------------------------------------------------------

def test_mesh_counts_table1():
    for row in read_golden("table1_mesh_counts.txt"):
        L = int(row["level"])
        if L > 3:
            continue
        w = mg.twisted_bar(L)
        assert w.nn == row["nodes"] and w.ne == row["elems"]
        assert int((w.dirichlet == 0).sum()) == row["free_dofs"]
    w = mg.twisted_bar(1)
    om = oracle.OracleMesh(w)
    free_nodes = w.dirichlet.reshape(-1, 3)[:, 0] == 0
    assert int(free_nodes.sum()) == 711
    assert int(om.patch_sizes()[free_nodes].sum()) == 7584


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_twisted_bar_table2(level):
    """J_grad of Benchmark 2 matches the printed Table 2 value to its 4 decimals."""
    row = [r for r in read_golden("table2_twisted_bar.txt") if int(r["level"]) == level][0]
    w = mg.twisted_bar(level)
    assert int((w.dirichlet == 0).sum()) == row["free_dofs"]
    om = oracle.OracleMesh(w)
    J, st = om.energy(w.v)
    assert st == oracle.OK
    assert abs(J - row["J_grad"]) <= 0.5e-4 + 1e-12


def test_twisted_bar_closed_form_and_convergence():
    """The continuum value alpha^2 C1 ly lz (ly^2+lz^2)/(12 lx) is printed as 6.326670; the
    P1 error shrinks by about 4 per uniform refinement (O(h^2))."""
    w1 = mg.twisted_bar(1)
    ex = w1.extra
    Jc = ex["alpha"] ** 2 * w1.C1 * ex["ly"] * ex["lz"] * (ex["ly"] ** 2 + ex["lz"] ** 2) / (12 * ex["lx"])
    # 6.32666949 is printed as 6.326670 (rounded twice: to 7, then 6 decimals)
    assert abs(Jc - 6.326670) < 1e-6
    errs = []
    for L in (1, 2, 3, 4):
        w = mg.twisted_bar(L)
        J, _ = oracle.OracleMesh(w).energy(w.v)
        errs.append(J - Jc)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(e > 0 for e in errs)
    assert all(3.5 < r < 4.5 for r in ratios), ratios


def _homog(w, A):
    X = w.coords
    return (X @ np.asarray(A).T).ravel()


@pytest.mark.parametrize("dim", [2, 3])
def test_neohooke_identity_zero_energy_and_gradient(dim):
    """W(I) = 0 and dW/dF(I) = 0 (eq. neoHook): with f = 0 and v = X, J = 0 and g = 0."""
    w = mg.neohooke_cube3d(4) if dim == 3 else mg.neohooke_rect2d(8, 4)
    w.f = None
    om = oracle.OracleMesh(w)
    v = w.coords.ravel().copy()
    J, st = om.energy(v)
    g, st2 = om.gradient_exact(v)
    assert st == st2 == oracle.OK
    assert J == 0.0
    assert np.abs(g).max() == 0.0


def test_neohooke_homogeneous_closed_forms():
    """Homogeneous deformations v = A X give F = A on every element, so J = W(A) |Omega|.
    Simple shear: det A = 1, I1 = dim + gamma^2, W = C1 gamma^2.
    Uniaxial stretch diag(s,1,1): W = C1 (s^2 - 1 - 2 log s) + D1 (s-1)^2."""
    w = _free_all(mg.neohooke_cube3d(4))
    w.f = None
    om = oracle.OracleMesh(w)
    C1, D1 = w.C1, w.D1
    gam = 0.3
    J, _ = om.energy(_homog(w, [[1, gam, 0], [0, 1, 0], [0, 0, 1]]))
    assert abs(J - C1 * gam ** 2) <= 1e-12 * C1 * gam ** 2
    s = 1.2
    J, _ = om.energy(_homog(w, np.diag([s, 1.0, 1.0])))
    ref = C1 * (s * s - 1 - 2 * math.log(s)) + D1 * (s - 1) ** 2
    assert abs(J - ref) <= 1e-12 * ref
    w2 = _free_all(mg.neohooke_rect2d(6, 3))
    w2.f = None
    om2 = oracle.OracleMesh(w2)
    J, _ = om2.energy(_homog(w2, [[1, gam], [0, 1]]))
    assert abs(J - 2.0 * C1 * gam ** 2) <= 1e-12 * C1        # |Omega| = 2


def test_neohooke_homogeneous_patch_test():
    """For F constant, sum_{T in patch(i)} |T| grad(phi_{T,i}) = 0 at every interior node,
    so the exact gradient vanishes at interior nodes and sums to zero over all nodes."""
    w = _free_all(mg.neohooke_cube3d(4))
    w.f = None
    om = oracle.OracleMesh(w)
    A = np.array([[1.1, 0.2, 0.0], [-0.1, 0.95, 0.05], [0.0, 0.1, 1.05]])
    g, st = om.gradient_exact(_homog(w, A))
    assert st == oracle.OK
    X = om.coords
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    scale = np.abs(g).max()
    assert np.abs(g.reshape(-1, 3)[interior]).max() <= 1e-12 * scale
    assert np.abs(g.reshape(-1, 3).sum(axis=0)).max() <= 1e-12 * scale


@pytest.mark.parametrize("p", [1.5, 2.0, 3.0])
def test_plaplace_linear_field(p):
    """v = a.x + c on every node gives J_grad = (1/p)|a|^p |Omega|; the unit square has
    |Omega| = 1."""
    w = _free_all(mg.plaplace_square(8, p=p))
    w.f = None
    om = oracle.OracleMesh(w)
    a = np.array([0.7, -1.3])
    J, _ = om.energy(om.coords @ a + 0.25)
    ref = np.linalg.norm(a) ** p / p
    assert abs(J - ref) <= 1e-13 * ref


def test_plaplace_p2_is_five_point_laplacian():
    """p = 2: the exact gradient is K v with K the P1 stiffness matrix, which on this
    right-triangle grid is the 5-point stencil 4 v_i - v_E - v_W - v_N - v_S at interior
    nodes; and J_grad = v.Kv/2."""
    n = 12
    w = mg.plaplace_square(n, p=2.0)
    w.f = None
    om = oracle.OracleMesh(w)
    V = w.v.reshape(n + 1, n + 1)
    g, st = om.gradient_exact(w.v)
    assert st == oracle.OK
    G = g.reshape(n + 1, n + 1)
    st5 = 4 * V[1:-1, 1:-1] - V[1:-1, 2:] - V[1:-1, :-2] - V[2:, 1:-1] - V[:-2, 1:-1]
    np.testing.assert_allclose(G[1:-1, 1:-1], st5, rtol=0, atol=1e-13)
    J, _ = om.energy(w.v)
    # v is zero on the boundary, so v.Kv only involves interior rows
    assert abs(J - 0.5 * float((V[1:-1, 1:-1] * st5).sum())) < 1e-12


@pytest.mark.parametrize("p", [1.5, 3.0])
def test_plaplace_euler_identity(p):
    """J_grad is positively homogeneous of degree p, so sum_n v_n dJ/dv_n = p J_grad."""
    w = _free_all(mg.plaplace_square(10, p=p))
    w.f = None
    om = oracle.OracleMesh(w)
    J, _ = om.energy(w.v)
    g, _ = om.gradient_exact(w.v)
    assert abs(g @ w.v - p * J) <= 1e-12 * p * J


def _rot3(a, b, c):
    ca, sa, cb, sb, cc, sc = map(float, (np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)))
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


def test_neohooke_frame_indifference_and_momentum():
    """W(RF) = W(F): J(Rv + c) = J(v).  Its derivatives: sum_i g_i = 0 (translations) and
    sum_i v_i x g_i = 0 (rotations), for the J_grad part with no dof removed."""
    w = _free_all(mg.random_small(3, 3, mg.MODEL_NEOHOOKE, 3, 3, 2))
    w.f = None
    om = oracle.OracleMesh(w)
    v = w.v
    R = _rot3(0.3, -0.7, 1.1)
    J0, _ = om.energy(v)
    J1, _ = om.energy((v.reshape(-1, 3) @ R.T + np.array([0.1, -2.0, 0.5])).ravel())
    assert abs(J1 - J0) <= 1e-11 * abs(J0)
    g, _ = om.gradient_exact(v)
    G = g.reshape(-1, 3)
    scale = np.abs(G).max() * np.abs(v).max()
    assert np.abs(G.sum(axis=0)).max() <= 1e-11 * np.abs(G).max()
    assert np.abs(np.cross(v.reshape(-1, 3), G).sum(axis=0)).max() <= 1e-11 * scale


# ---------------------------------------------------------------------------------
# Exact gradient (Sec. 6.2): derivatives taken independently
# ---------------------------------------------------------------------------------

def _complex_energy(om, vc):
    """J_grad(v) in complex arithmetic from the oracle's (separately pinned) dphi, vol."""
    dim, d, k = om.dim, om.d, om.dim + 1
    G = om.dphi.reshape(om.ne, k, dim)
    U = vc.reshape(om.nn, d)
    if om.model == oracle.NEOHOOKE:
        U = U - om.coords
    Ue = U[om.elems]                                        # ne x k x d
    F = np.einsum("ekj,ekm->ejm", Ue, G)
    if om.model == oracle.NEOHOOKE:
        F = F + np.eye(dim)[None]
        I1 = (F * F).sum(axis=(1, 2))
        det = np.linalg.det(F)
        W = om.C1 * (I1 - dim - 2 * np.log(det)) + om.D1 * (det - 1) ** 2
    else:
        s = (F[:, 0, :] ** 2).sum(axis=1)
        W = s ** (om.p / 2) / om.p
    return (om.vol * W).sum()


@pytest.mark.parametrize("dim,model", [(2, mg.MODEL_PLAPLACE), (2, mg.MODEL_NEOHOOKE),
                                       (3, mg.MODEL_NEOHOOKE)])
def test_exact_gradient_matches_complex_step(dim, model):
    """Complex-step differentiation (Squire & Trapp 1998): dJ/dv_n = Im J(v + i h e_n)/h
    to machine precision with h = 1e-30, independent of the hand-derived dW/dF."""
    w = _free_all(mg.random_small(11, dim, model, 3, 2, 2))
    w.f = None
    om = oracle.OracleMesh(w)
    g, st = om.gradient_exact(w.v)
    assert st == oracle.OK
    h = 1e-30
    cs = np.empty_like(g)
    for n in range(g.shape[0]):
        vc = w.v.astype(np.complex128)
        vc[n] += 1j * h
        cs[n] = _complex_energy(om, vc).imag / h
    np.testing.assert_allclose(g, cs, rtol=0, atol=1e-12 * np.abs(cs).max())


def _global_cd(om, v, eps, dofs):
    out = []
    for n in dofs:
        vp = v.copy(); vp[n] += eps
        vm = v.copy(); vm[n] -= eps
        out.append((om.energy(vp)[0] - om.energy(vm)[0]) / (2 * eps))
    return np.array(out)


@pytest.mark.parametrize("dim,model", [(2, mg.MODEL_PLAPLACE), (3, mg.MODEL_NEOHOOKE)])
def test_exact_gradient_vs_central_differences_order2(dim, model):
    """Central differences of the energy converge to the exact gradient as O(eps^2)
    (eq. CD): halving eps divides the error by about 4."""
    w = mg.random_small(17, dim, model, 3, 3, 2)
    om = oracle.OracleMesh(w)
    g, _ = om.gradient_exact(w.v)
    free = np.flatnonzero(w.dirichlet == 0)[:12]
    h = 1.0 / 3
    base = 0.02 if model == mg.MODEL_NEOHOOKE else 0.05
    errs = []
    for eps in (base * h, base * h / 2):
        cd = _global_cd(om, w.v, eps, free)     # J includes -b.v
        errs.append(np.abs(cd - g[free]).max())
    assert errs[1] < errs[0]
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


@pytest.mark.parametrize("dim,model", [(2, mg.MODEL_PLAPLACE), (2, mg.MODEL_NEOHOOKE),
                                       (3, mg.MODEL_NEOHOOKE)])
def test_patch_cd_equals_global_cd(dim, model):
    """Only the elements of the patch of dof n change when v_n moves (eqs. CDS, sumpatch),
    so the patch-local central difference equals the global one up to rounding."""
    w = mg.random_small(23, dim, model, 3, 3, 2)
    om = oracle.OracleMesh(w)
    eps = 1e-4
    free = np.flatnonzero(w.dirichlet == 0)
    gp, st = om.gradient_fd(w.v, eps, free)
    assert st == oracle.OK
    gg = _global_cd(om, w.v, eps, free)     # J includes -b.v
    Jabs = np.abs(om.vol * om.energy(w.v, densities=True)[2]).sum()
    tol = 64 * 2.2e-16 * Jabs / eps + 1e-12 * np.abs(gg).max()
    assert np.abs(gp - gg).max() <= tol


def test_patch_fd_all_dofs_matches_subset_and_zero_on_dirichlet():
    w = mg.plaplace_square(8)
    om = oracle.OracleMesh(w)
    gall, st = om.gradient_fd(w.v, 1e-6)
    assert st == oracle.OK
    assert np.all(gall[w.dirichlet == 1] == 0.0)
    sub = np.array([10, 40, 41, 70], dtype=np.int64)
    gs, _ = om.gradient_fd(w.v, 1e-6, sub)
    np.testing.assert_array_equal(gs, gall[sub])


@pytest.mark.parametrize("dim,model", [(2, mg.MODEL_PLAPLACE), (3, mg.MODEL_NEOHOOKE)])
def test_patch_fd_converges_to_exact(dim, model):
    w = mg.random_small(29, dim, model, 4, 3, 2)
    om = oracle.OracleMesh(w)
    g, _ = om.gradient_exact(w.v)
    free = np.flatnonzero(w.dirichlet == 0)
    e1 = np.abs(om.gradient_fd(w.v, 4e-3, free)[0] - g[free]).max()
    e2 = np.abs(om.gradient_fd(w.v, 2e-3, free)[0] - g[free]).max()
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_gradient_includes_minus_b_and_zero_dirichlet():
    """grad J = grad J_grad - b on free dofs (eq. linearTermGrad) and 0 on Dirichlet dofs."""
    w = mg.plaplace_square(8)
    om = oracle.OracleMesh(w)
    g, _ = om.gradient_exact(w.v)
    assert np.all(g[w.dirichlet == 1] == 0.0)
    b = om.b.copy()
    om.set_load(None)
    g0, _ = om.gradient_exact(w.v)
    free = w.dirichlet == 0
    np.testing.assert_allclose(g[free], g0[free] - b[free], atol=1e-15)
    J0, _ = om.energy(w.v)
    om.b = b
    J1, _ = om.energy(w.v)
    assert abs((J0 - J1) - b @ w.v) < 1e-13


def test_inverted_element_reports_domain_error():
    w = mg.neohooke_cube3d(3)
    om = oracle.OracleMesh(w)
    v = w.coords.ravel().copy()
    v[3 * 21 + 0] += 2.0                  # fold one interior node far past its neighbours
    J, st = om.energy(v)
    assert st == oracle.EDOMAIN and J == math.inf
    _, st = om.gradient_exact(v)
    assert st == oracle.EDOMAIN
