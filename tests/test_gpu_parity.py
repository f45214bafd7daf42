"""GPU (libfemenergy.so, through the C ABI) against the CPU oracle, element by element.

Sizes span several 256-thread tiles with ragged tails; the full-size workloads are the
2D p-Laplacian 64x64x2, the 2D Neo-Hookean 1024x512x2 and the 3D Neo-Hookean 128^3x6 mesh,
run in the same launch configuration the benchmark times.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import (check_energy, check_grad, energy_scale, fd_extra)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fem():
    from paper_2109_01158_gb300 import fem
    return fem


def _gpu(w, **kw):
    return _fem().FEMesh.from_workload(w, **kw)


def _v(w):
    return torch.from_numpy(np.ascontiguousarray(w.v)).cuda()


# ----------------------------------------------------------------------------------------
# a1: precompute, patches, load vector
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("maker", [
    lambda: mg.random_small(1, 2, mg.MODEL_PLAPLACE, 23, 17),
    lambda: mg.random_small(2, 3, mg.MODEL_NEOHOOKE, 9, 7, 5),
    lambda: mg.twisted_bar(1),
])
@pytest.mark.parametrize("order", [0, 1])
def test_precompute_patches_and_load_vector(maker, order):
    w = maker()
    if w.f is None:
        w.f = mg.uniform(99, np.arange(w.ndof), -1, 1)
    om = oracle.OracleMesh(w)
    gm = _gpu(w, order=order)
    dphi, vol = gm.shape_gradients()
    # the precompute uses the same correctly rounded operations as the oracle
    np.testing.assert_array_equal(vol, om.vol)
    np.testing.assert_array_equal(dphi, om.dphi)
    row_ptr, ent = gm.patches()
    np.testing.assert_array_equal(row_ptr, om.row_ptr)
    np.testing.assert_array_equal(ent, om.ent)
    b = gm.load_vector()
    # b_i is a sum over the patch of node i; the device keeps the elements in Morton order of
    # their centroids, so the patch sums run in another order than the oracle's
    np.testing.assert_allclose(b, om.b, rtol=1e-13, atol=1e-15 * np.abs(om.b).max())


# ----------------------------------------------------------------------------------------
# a2-a6: energy and exact gradient, FP64
# ----------------------------------------------------------------------------------------

def _parity(w, order=0, check_dens=True, precision=0):
    om = oracle.OracleMesh(w)
    gm = _gpu(w, order=order, precisions=(precision,))
    v = _v(w)
    J, dens = gm.energy(v, densities=True)
    Jg, g = gm.energy_gradient(v)
    g2 = gm.gradient_exact(v)
    assert gm.sync_status() == 0
    Jref, st, dref = om.energy(w.v, densities=True)
    gref, st2 = om.gradient_exact(w.v)
    assert st == st2 == oracle.OK
    scale = energy_scale(om, w.v)
    e1 = check_energy(J.item(), Jref, scale)
    check_energy(Jg.item(), Jref, scale)
    e2 = check_grad(g.cpu().numpy(), gref)
    np.testing.assert_array_equal(g.cpu().numpy(), g2.cpu().numpy())
    assert Jg.item() == J.item()
    if check_dens:
        np.testing.assert_allclose(dens.cpu().numpy(), dref, rtol=1e-9,
                                   atol=1e-12 * np.abs(dref).max())
    return e1, e2


@pytest.mark.parametrize("seed,dim,model,n", [
    (1, 2, mg.MODEL_PLAPLACE, (13, 11)), (2, 2, mg.MODEL_NEOHOOKE, (19, 23)),
    (3, 3, mg.MODEL_NEOHOOKE, (7, 5, 9)), (4, 3, mg.MODEL_PLAPLACE, (6, 6, 5)),
    (5, 2, mg.MODEL_NEOHOOKE, (1, 1)), (6, 3, mg.MODEL_NEOHOOKE, (1, 1, 1)),
])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_random_meshes(seed, dim, model, n, order, precision):
    w = mg.random_small(seed, dim, model, *n)
    _parity(w, order, precision=precision)


@pytest.mark.parametrize("p", [1.5, 2.0, 3.0, 4.0, 4.5])
@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_plaplace_exponents(p, precision):
    w = mg.plaplace_square(17, p=p)
    _parity(w, precision=precision)


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_c1_plaplace_64(precision):
    _parity(mg.plaplace_square(64), precision=precision)


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_shuffled_nodes_3d(precision):
    w = mg.shuffle_nodes(mg.neohooke_cube3d(9), seed=4)
    _parity(w, order=0, precision=precision)
    _parity(w, order=1, precision=precision)
    _parity(w, order=2, precision=precision)


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_c2_neohooke_2d_full(precision):
    """2D Neo-Hookean 1024x512x2 (1,048,576 triangles) with the benchmark's launch shape."""
    w = mg.neohooke_rect2d()
    e1, e2 = _parity(w, check_dens=False, precision=precision)
    print(f"C2 precision {precision}: energy err/condition {e1:.2e}, gradient rel {e2:.2e}")


def test_c2_literal_noise_folds_the_same_elements():
    """With U[-1e-3,1e-3] noise (51% of the spacing) the 1024x512x2 mesh folds: GPU and oracle
    find exactly the same inverted triangles (W = +Inf), J = +Inf and FE_EDOMAIN."""
    fem = _fem()
    w = mg.neohooke_rect2d(noise=1e-3)
    om = oracle.OracleMesh(w)
    Jref, st, dref = om.energy(w.v, densities=True)
    assert st == oracle.EDOMAIN and Jref == math.inf
    gm = _gpu(w)
    J, dens = gm.energy(_v(w), densities=True)
    assert gm.sync_status() == fem.FE_EDOMAIN
    assert J.item() == math.inf
    bad_gpu = np.isinf(dens.cpu().numpy())
    np.testing.assert_array_equal(bad_gpu, np.isinf(dref))
    assert int(bad_gpu.sum()) == 28819


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_c3_neohooke_3d_full(precision):
    """3D Neo-Hookean 128^3 x 6 (12,582,912 tetrahedra), energy and exact gradient against
    the oracle on every dof, in the launch configuration of the benchmark."""
    w = mg.neohooke_cube3d(128)
    e1, e2 = _parity(w, check_dens=False, precision=precision)
    print(f"C3 precision {precision}: energy err/condition {e1:.2e}, gradient rel {e2:.2e}")


def _w_homogeneous_decimal(A, C1, D1):
    """W(A) of eq. neoHook for a 3x3 matrix A in 50-digit decimal arithmetic."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    a = [[Decimal(repr(float(x))) for x in row] for row in A]
    det = (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
           + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
    I1 = sum(x * x for row in a for x in row)
    W = Decimal(repr(C1)) * (I1 - 3 - 2 * det.ln()) + Decimal(repr(D1)) * (det - 1) ** 2
    return float(W)


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_small_strain_homogeneous_energy(precision, eps):
    """Small strains: v = (I + eps B) X on the unit cube gives J = W(I + eps B) exactly.  The
    kernels evaluate eq. neoHook in displacement form and keep full relative accuracy even
    where I1 - 3 - 2 log det F cancels down to O(eps^2) (the formula as written loses about
    1e-16 / eps^2 relative); reference in 50-digit decimals.  The tolerance adds the rounding
    of the input itself: v = X + u is stored in FP64 with |v| ~ 1, so u carries a relative
    error of about 1e-16 / eps and W ~ u^2 twice that."""
    fem = _fem()
    w = mg.neohooke_cube3d(6)
    w.dirichlet[:] = 0
    w.f = None
    B = np.array([[0.3, -0.2, 0.1], [0.05, -0.4, 0.2], [-0.1, 0.25, 0.15]])
    A = np.eye(3) + eps * B
    w.v = (w.coords @ A.T).ravel()
    ref = _w_homogeneous_decimal(A, w.C1, w.D1)
    gm = _gpu(w, precisions=(precision,))
    J = gm.energy(_v(w)).item()
    assert abs(J - ref) <= (1e-12 + 4.4e-16 / eps) * abs(ref), (J, ref)


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
@pytest.mark.parametrize("delta", [-0.25, -0.1, -0.0021, 0.0019, 0.003, 0.05, 0.3, 0.42, 0.6])
def test_homogeneous_stretch_energy_over_the_log_range(precision, delta):
    """v = A X with A = (1 + delta)^(1/3) (I + 0.02 S) (det A - 1 = delta up to O(0.02^2)):
    J = W(A) on the unit cube.  The values of det F - 1 cover the breakpoint table of
    phi(x) = x - log(1 + x) of the FP64 kernels on both sides of zero, next to the +-1/512 row
    boundaries, and beyond it (0.6: the log1p branch); reference in 50-digit decimals."""
    fem = _fem()
    w = mg.neohooke_cube3d(6)
    w.dirichlet[:] = 0
    w.f = None
    S = np.array([[0.0, 0.3, -0.1], [0.2, 0.0, 0.25], [-0.15, 0.1, 0.0]])
    A = (1.0 + delta) ** (1.0 / 3.0) * (np.eye(3) + 0.02 * S)
    w.v = (w.coords @ A.T).ravel()
    ref = _w_homogeneous_decimal(A, w.C1, w.D1)
    gm = _gpu(w, precisions=(precision,))
    J = gm.energy(_v(w)).item()
    # input rounding of v = A X (~1e-16 of |v|, averaging over the elements) enters W
    # through dW/dF ~ C1 |F| + D1
    tol = 1e-12 * abs(ref) + 1e-16 * (w.C1 + w.D1)
    assert abs(J - ref) <= tol, (J, ref, abs(J - ref) / abs(ref))


def test_twisted_bar_df64_levels():
    """Double-float energies of Benchmark 2 (E = 2e8, volumes down to 1e-10) against the
    oracle at the FP64 tolerance, levels 1-4."""
    fem = _fem()
    for level in (1, 2, 3, 4):
        w = mg.twisted_bar(level)
        om = oracle.OracleMesh(w)
        gm = _gpu(w, precisions=(fem.FE_DF64,))
        J, g = gm.energy_gradient(_v(w))
        check_energy(J.item(), om.energy(w.v)[0], energy_scale(om, w.v))
        check_grad(g.cpu().numpy(), om.gradient_exact(w.v)[0])


def test_df64_log_accuracy():
    """The double-float logarithm of the FE_DF64 kernels against numpy's FP64 log:
    |y - log x| <= 2^-45 |log x| + 2^-51 over 12 decades and around 1."""
    fem = _fem()
    w = mg.neohooke_cube3d(2)
    gm = _gpu(w, precisions=(fem.FE_DF64,))
    u = mg.uniform(5, np.arange(200000), 0.0, 1.0)
    x = np.concatenate([10.0 ** (12 * u - 6), 1.0 + (u - 0.5) * 1e-3, 1.0 + (u - 0.5) * 1e-9,
                        0.5 + 1.5 * u, [1.0, 2.0, 0.5, 1.4142135, 0.70710678, 1.0 + 2.0 ** -30]])
    y = gm.diag_df64_log(torch.from_numpy(x)).cpu().numpy()
    # the input itself is first rounded to a double-float (hi + lo): compare with its log
    hi = x.astype(np.float32).astype(np.float64)
    xr = hi + (x - hi).astype(np.float32).astype(np.float64)
    ref = np.log(xr)
    # k ln2, the table value and log(1+t) are combined by three double-word sums and one
    # product, each within about 2^-48 relative: 2^-45 |log x| bounds their sum
    err = np.abs(y - ref) / (2.0 ** -45 * np.abs(ref) + 2.0 ** -51)
    assert err.max() <= 1.0, (err.max(), x[err.argmax()])


def test_twisted_bar_matches_table2():
    """The GPU reproduces Benchmark 2 Table 2 (levels 1-3) to the printed 4 decimals."""
    for level, ref in [(1, 12.6623), (2, 7.9083), (3, 6.7219)]:
        w = mg.twisted_bar(level)
        J = _gpu(w).energy(_v(w)).item()
        assert abs(J - ref) <= 0.5e-4


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["f64", "f32", "df64"])
def test_deterministic_bitwise(precision):
    w = mg.neohooke_cube3d(24)
    gm = _gpu(w, precisions=(precision,))
    v = _v(w)
    J1, g1 = gm.energy_gradient(v)
    J2, g2 = gm.energy_gradient(v)
    assert J1.item() == J2.item()
    assert torch.equal(g1, g2)


# ----------------------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------------------

def test_no_elements_and_all_dirichlet():
    w = mg.plaplace_square(4)
    w0 = mg.Workload("empty", 2, 1, w.coords, np.zeros((0, 3), np.int32), w.dirichlet,
                     mg.MODEL_PLAPLACE, p=3.0, f=None, v=w.v)
    gm = _gpu(w0)
    J, g = gm.energy_gradient(_v(w0))
    assert J.item() == 0.0 and float(g.abs().max()) == 0.0
    w.dirichlet[:] = 1
    om = oracle.OracleMesh(w)
    J, g = _gpu(w).energy_gradient(_v(w))
    assert float(g.abs().max()) == 0.0
    check_energy(J.item(), om.energy(w.v)[0], energy_scale(om, w.v))


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["f64", "f32", "df64"])
def test_inverted_element_reports_domain_error(precision):
    fem = _fem()
    w = mg.neohooke_cube3d(3)
    v = w.coords.ravel().copy()
    v[3 * 21] += 2.0
    w.v = v
    gm = _gpu(w, precisions=(precision,))
    J = gm.energy(_v(w))
    assert gm.sync_status() == fem.FE_EDOMAIN
    assert J.item() == math.inf
    assert gm.sync_status() == fem.FE_OK         # status is cleared
    _, _, st = gm.energy_gradient_host(w.v)
    assert st == fem.FE_EDOMAIN


def test_bad_arguments_are_rejected():
    fem = _fem()
    w = mg.plaplace_square(4)
    with pytest.raises(fem.FEError):
        fem.FEMesh(2, 1, w.coords, np.array([[0, 1, 99]], np.int32), model=fem.FE_PLAPLACE, p=3.0)
    with pytest.raises(fem.FEError):
        fem.FEMesh(2, 1, w.coords, np.array([[0, 1, 1]], np.int32), model=fem.FE_PLAPLACE, p=3.0)
    with pytest.raises(fem.FEError):   # Neo-Hookean needs d = dim
        fem.FEMesh(2, 1, w.coords, w.elems, model=fem.FE_NEOHOOKE, C1=1.0, D1=1.0)
    with pytest.raises(fem.FEError):   # degenerate element
        c = np.array([[0, 0], [1, 0], [2, 0]], float)
        fem.FEMesh(2, 1, c, np.array([[0, 1, 2]], np.int32), model=fem.FE_PLAPLACE, p=3.0)
    gm = _gpu(w)
    with pytest.raises(fem.FEError):
        gm.gradient_fd(_v(w), -1.0)


# ----------------------------------------------------------------------------------------
# a7: central differences over patches
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed,dim,model,n", [
    (7, 2, mg.MODEL_PLAPLACE, (9, 7)), (8, 2, mg.MODEL_NEOHOOKE, (8, 9)),
    (9, 3, mg.MODEL_NEOHOOKE, (4, 5, 3)),
])
@pytest.mark.parametrize("order", [0, 1])
def test_fd_patch_gradient(seed, dim, model, n, order):
    w = mg.random_small(seed, dim, model, *n)
    om = oracle.OracleMesh(w)
    gm = _gpu(w, order=order)
    eps = 1e-6
    gref, _ = om.gradient_fd(w.v, eps)
    extra = fd_extra(om, w.v, eps)
    check_grad(gm.gradient_fd(_v(w), eps).cpu().numpy(), gref, extra_abs=extra)
    dofs = np.array([0, 3, w.ndof - 1, 5, 3], dtype=np.int64)
    gs = gm.gradient_fd(_v(w), eps, dofs).cpu().numpy()
    check_grad(gs, om.gradient_fd(w.v, eps, dofs)[0], extra_abs=extra)


def test_c1_fd_full():
    """2D p-Laplacian 64x64x2: central-difference gradient on every dof, eps = 1e-6."""
    w = mg.plaplace_square(64)
    om = oracle.OracleMesh(w)
    g = _gpu(w).gradient_fd(_v(w), 1e-6).cpu().numpy()
    gref, _ = om.gradient_fd(w.v, 1e-6)
    check_grad(g, gref, extra_abs=fd_extra(om, w.v, 1e-6))


def test_c3_fd_subset_10k():
    """3D Neo-Hookean 128^3x6: central differences on 10^4 random free dofs (seed 2)
    against the oracle, and against the exact gradient within O(eps^2) + rounding."""
    w = mg.neohooke_cube3d(128)
    free = np.flatnonzero(w.dirichlet == 0)
    pick = np.argsort(mg.splitmix64(2, np.arange(free.size)))[:10000]
    dofs = free[np.sort(pick)].astype(np.int64)
    om = oracle.OracleMesh(w)
    gm = _gpu(w)
    v = _v(w)
    g = gm.gradient_fd(v, 1e-6, dofs).cpu().numpy()
    gref, _ = om.gradient_fd(w.v, 1e-6, dofs)
    extra = fd_extra(om, w.v, 1e-6)
    check_grad(g, gref, extra_abs=extra)
    gex = gm.gradient_exact(v).cpu().numpy()[dofs]
    check_grad(g, gex, rtol=1e-6, extra_abs=extra)


def test_c3_fd_full_matches_subset_and_exact():
    """3D Neo-Hookean 128^3x6: the central-difference gradient on every dof (full mode, which
    updates the terms of the density per perturbed row) agrees with the oracle's central
    differences (eqs. CD / CDS, each perturbed density rebuilt from its perturbed row) on 10^4
    random free dofs, with the GPU's subset mode on the same dofs, and with the exact gradient
    within O(eps^2) + rounding."""
    w = mg.neohooke_cube3d(128)
    free = np.flatnonzero(w.dirichlet == 0)
    dofs = free[np.sort(np.argsort(mg.splitmix64(3, np.arange(free.size)))[:10000])].astype(np.int64)
    om = oracle.OracleMesh(w)
    gm = _gpu(w)
    v = _v(w)
    full = gm.gradient_fd(v, 1e-6).cpu().numpy()
    assert gm.sync_status() == 0
    extra = fd_extra(om, w.v, 1e-6)
    gref, st = om.gradient_fd(w.v, 1e-6, dofs)
    assert st == oracle.OK
    gref = np.asarray(gref)
    err = float(np.abs(full[dofs] - gref).max())
    print(f"C3 full-mode CD vs oracle CD on 1e4 dofs: max |diff| {err:.3e}, "
          f"bar {1e-10 * float(np.abs(gref).max()) + extra:.3e} (||g*|| {float(np.abs(gref).max()):.3e})")
    check_grad(full[dofs], gref, extra_abs=extra)
    check_grad(full[dofs], gm.gradient_fd(v, 1e-6, dofs).cpu().numpy(), extra_abs=extra)
    check_grad(full, gm.gradient_exact(v).cpu().numpy(), rtol=1e-6, extra_abs=extra)
    assert np.all(full[w.dirichlet != 0] == 0.0)


def test_fd_small_strain_matches_exact_gradient():
    """Near F = I (displacements of 1e-6, eps = 1e-7) the patch energies are evaluated in
    displacement form, so their rounding is relative to W, not to the O(1) terms of the
    formula as written: the central differences then agree with the exact gradient to their
    O(eps^2) truncation (~1e-9 relative here), where differences of the formula as written
    would carry ~u C1 dim |T| / eps ~ 5e-6 relative of rounding."""
    w = mg.neohooke_cube3d(8)
    w.v = w.coords.ravel() + mg.uniform(11, np.arange(w.ndof), -1e-6, 1e-6) * (w.dirichlet == 0)
    gm = _gpu(w)
    v = _v(w)
    g = gm.gradient_exact(v).cpu().numpy()
    gfd = gm.gradient_fd(v, 1e-7).cpu().numpy()
    check_grad(gfd, g, rtol=1e-8)
    dofs = np.flatnonzero(w.dirichlet == 0)[::7].astype(np.int64)
    check_grad(gm.gradient_fd(v, 1e-7, dofs).cpu().numpy(), g[dofs], rtol=1e-8)


# ----------------------------------------------------------------------------------------
# a8: autograd
# ----------------------------------------------------------------------------------------

def test_autograd_backward_is_exact_gradient():
    fem = _fem()
    w = mg.random_small(31, 3, mg.MODEL_NEOHOOKE, 5, 4, 3)
    gm = _gpu(w)
    v = _v(w).requires_grad_(True)
    J = fem.energy(v, gm)
    J.backward()
    gref, _ = oracle.OracleMesh(w).gradient_exact(w.v)
    check_grad(v.grad.cpu().numpy(), gref)
    v.grad = None
    (3.0 * fem.energy(v, gm)).backward()
    check_grad(v.grad.cpu().numpy(), 3.0 * gref)


def test_autograd_gradcheck_free_dofs():
    fem = _fem()
    w = mg.random_small(37, 2, mg.MODEL_NEOHOOKE, 3, 2)
    gm = _gpu(w)
    free = torch.from_numpy(np.flatnonzero(w.dirichlet == 0)).cuda()
    base = _v(w)

    def f(x):
        full = base.clone().index_put((free,), x)
        return fem.energy(full, gm)

    x = base[free].clone().requires_grad_(True)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-5, rtol=1e-4)


# ----------------------------------------------------------------------------------------
# a9: FP32 element arithmetic with compensated reductions
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("maker,jtol,gtol", [
    (lambda: mg.neohooke_rect2d(256, 128), 2e-6, 2e-5),
    (lambda: mg.neohooke_cube3d(32), 2e-6, 2e-5),
    (lambda: mg.plaplace_square(64), 2e-6, 2e-5),
    (lambda: mg.neohooke_cube3d(128), 2e-6, 2e-5),
])
def test_fp32_compensated_error(maker, jtol, gtol):
    fem = _fem()
    w = maker()
    om = oracle.OracleMesh(w)
    gm = _gpu(w, precisions=(fem.FE_F32_COMP, fem.FE_F64))
    assert gm.precision == fem.FE_F32_COMP
    J, g = gm.energy_gradient(_v(w))
    Jref, _ = om.energy(w.v)
    gref, _ = om.gradient_exact(w.v)
    ej = check_energy(J.item(), Jref, energy_scale(om, w.v), rtol=jtol)
    eg = check_grad(g.cpu().numpy(), gref, rtol=gtol)
    print(f"{w.name}: FP32-comp energy err/condition {ej:.2e}, gradient rel {eg:.2e}")
    assert eg > 1e-12, "the FP32 path returned FP64-accurate gradients: wrong kernel ran"
    gm.set_precision(fem.FE_F64)
    J64, _ = gm.energy_gradient(_v(w))
    check_energy(J64.item(), Jref, energy_scale(om, w.v))


# ----------------------------------------------------------------------------------------
# end-to-end host call
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_host_call_matches_device_call(pinned, precision):
    """fe_energy_gradient_host (staged copies for pageable buffers; kernels reading v and
    writing g in page-locked host memory directly) gives bitwise the device call's J and g."""
    w = mg.neohooke_cube3d(16)
    gm = _gpu(w, precisions=(precision,))
    J, g = gm.energy_gradient(_v(w))
    if pinned:
        vt = torch.from_numpy(w.v).pin_memory()
        gt = torch.zeros(w.ndof, dtype=torch.float64).pin_memory()
        Jh, gh, st = gm.energy_gradient_host(vt.numpy(), gt.numpy())
    else:
        Jh, gh, st = gm.energy_gradient_host(w.v)
    assert st == 0
    assert Jh == J.item()
    np.testing.assert_array_equal(gh, g.cpu().numpy())
