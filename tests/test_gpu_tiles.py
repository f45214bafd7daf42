"""The fused element + patch kernels (element tiles with the local forces in shared memory;
FE_F32_COMP) against the CPU oracle, through the C ABI.

Beyond the workloads of test_gpu_parity.py these meshes exercise the tile structure itself:
every node order and both vector numberings, a fan whose centre node lies in every element
(its patch spans many tiles, so its gradient is the sum of many tile partials), disjoint
elements (tiles cut by the node limit), nodes that belong to no element (node-only tiles,
g = -b there), empty meshes, and the bitwise agreement of the energy-only, gradient-only and
fused calls.  Bars: the FP32 path's stated errors, 2e-6 of the energy's condition number and
2e-5 of ||g*||_inf (the measured error is printed per result)."""
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, check_grad, energy_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JTOL, GTOL = 2e-6, 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fem():
    from paper_2109_01158_gb300 import fem
    return fem


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _tile_parity(w, precision, order=0, device_vectors=False, dens_rtol=2e-5):
    """Energy (with densities), energy + gradient and gradient alone against the oracle; the
    three calls agree bitwise on what they share."""
    fem = _fem()
    om = oracle.OracleMesh(w)
    gm = fem.FEMesh.from_workload(w, order=order, precisions=(precision,))
    v = _dev(w.v)
    if device_vectors:
        gm.set_vector_order(fem.FE_VECTORS_DEVICE)
        v = gm.to_device_order(v)
    J, dens = gm.energy(v, densities=True)
    Jg, g = gm.energy_gradient(v)
    g2 = gm.gradient_exact(v)
    assert gm.sync_status() == fem.FE_OK
    if device_vectors:
        g = gm.from_device_order(g)
        g2 = gm.from_device_order(g2)
    Jref, st, dref = om.energy(w.v, densities=True)
    gref, st2 = om.gradient_exact(w.v)
    assert st == st2 == oracle.OK
    scale = energy_scale(om, w.v)
    ej = check_energy(J.item(), Jref, scale, rtol=JTOL)
    assert Jg.item() == J.item()
    eg = check_grad(g.cpu().numpy(), gref, rtol=GTOL)
    np.testing.assert_array_equal(g.cpu().numpy(), g2.cpu().numpy())
    d = dens.cpu().numpy()
    np.testing.assert_allclose(d, dref, rtol=dens_rtol, atol=dens_rtol * max(np.abs(dref).max(), 1e-300))
    print(f"{w.name} order {order}: energy err/condition {ej:.2e}, gradient rel {eg:.2e}")
    return ej, eg


@pytest.mark.parametrize("seed,dim,model,n", [
    (1, 2, mg.MODEL_PLAPLACE, (13, 11)), (2, 2, mg.MODEL_NEOHOOKE, (19, 23)),
    (3, 3, mg.MODEL_NEOHOOKE, (7, 5, 9)), (4, 3, mg.MODEL_PLAPLACE, (6, 6, 5)),
    (5, 2, mg.MODEL_NEOHOOKE, (1, 1)), (6, 3, mg.MODEL_NEOHOOKE, (1, 1, 1)),
    (11, 3, mg.MODEL_NEOHOOKE, (17, 13, 11)), (12, 2, mg.MODEL_PLAPLACE, (61, 47)),
])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_random_meshes_f32(seed, dim, model, n, order):
    w = mg.random_small(seed, dim, model, *n)
    _tile_parity(w, _fem().FE_F32_COMP, order)


@pytest.mark.parametrize("p", [1.5, 2.0, 3.0, 4.5])
def test_plaplace_exponents_f32(p):
    _tile_parity(mg.plaplace_square(33, p=p), _fem().FE_F32_COMP)


def test_device_vector_order_and_shuffled_nodes_f32():
    w = mg.shuffle_nodes(mg.neohooke_cube3d(12), seed=4)
    for order in (0, 1, 2):
        _tile_parity(w, _fem().FE_F32_COMP, order, device_vectors=(order == 1))


def _fan(n_tri, seed=21):
    """2D p-Laplacian on a fan of n_tri triangles around the origin: the centre node is in
    every element, so its patch spans every tile."""
    ang = 2 * np.pi * np.arange(n_tri) / n_tri
    rad = 1.0 + 0.3 * mg.uniform(seed, np.arange(n_tri), 0.0, 1.0)
    coords = np.vstack([[0.0, 0.0], np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)])
    k = np.arange(n_tri)
    elems = np.stack([np.zeros(n_tri, np.int64), 1 + k, 1 + (k + 1) % n_tri], axis=1).astype(np.int32)
    nn = coords.shape[0]
    dirichlet = np.zeros(nn, np.uint8)
    dirichlet[1::7] = 1
    return mg.Workload(f"fan{n_tri}", 2, 1, coords, elems, dirichlet, mg.MODEL_PLAPLACE, p=3.0,
                       f=mg.uniform(seed + 1, np.arange(nn), -1.0, 1.0),
                       v=mg.uniform(seed + 2, np.arange(nn), -1.0, 1.0))


def test_fan_centre_node_spans_many_tiles_f32():
    _tile_parity(_fan(5000), _fem().FE_F32_COMP)


def _disjoint_tets(n, seed=31):
    """n tetrahedra sharing no node (each tile is cut by the node limit, not the element
    count), plus 37 nodes in no element."""
    rng_c = mg.uniform(seed, np.arange(n * 3), 0.0, 1.0).reshape(n, 3) * 10.0
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.3
    coords = (rng_c[:, None, :] + ref[None, :, :]).reshape(-1, 3)
    extra = mg.uniform(seed + 1, np.arange(37 * 3), 0.0, 10.0).reshape(37, 3)
    coords = np.vstack([coords, extra])
    elems = np.arange(4 * n, dtype=np.int32).reshape(n, 4)
    nn = coords.shape[0]
    C1, D1 = mg.lame_c1_d1(1e4, 0.3)
    v = coords.ravel() + mg.uniform(seed + 2, np.arange(nn * 3), -0.01, 0.01)
    dirichlet = (mg.uniform(seed + 3, np.arange(nn * 3), 0.0, 1.0) < 0.1).astype(np.uint8)
    return mg.Workload(f"disjoint{n}", 3, 3, coords, elems, dirichlet, mg.MODEL_NEOHOOKE, C1=C1, D1=D1,
                       f=mg.uniform(seed + 4, np.arange(nn * 3), -1.0, 1.0), v=v)


def test_disjoint_elements_and_isolated_nodes_f32():
    _tile_parity(_disjoint_tets(3000), _fem().FE_F32_COMP)


def test_empty_and_nodes_only_f32():
    fem = _fem()
    w = mg.plaplace_square(9)
    w.f = mg.uniform(5, np.arange(w.nn), -1.0, 1.0)
    w0 = mg.Workload("nodes-only", 2, 1, w.coords, np.zeros((0, 3), np.int32), w.dirichlet,
                     mg.MODEL_PLAPLACE, p=3.0, f=w.f, v=w.v)
    om = oracle.OracleMesh(w0)
    gm = fem.FEMesh.from_workload(w0, precisions=(fem.FE_F32_COMP,))
    J, g = gm.energy_gradient(_dev(w0.v))
    gref, _ = om.gradient_exact(w0.v)
    Jref, _ = om.energy(w0.v)
    check_energy(J.item(), Jref, energy_scale(om, w0.v), rtol=1e-15)
    np.testing.assert_array_equal(g.cpu().numpy(), gref)


def test_inverted_element_gives_inf_f32():
    fem = _fem()
    w = mg.neohooke_cube3d(10)
    v = w.coords.ravel().copy()
    v[3 * 100] += 2.0
    w.v = v
    gm = fem.FEMesh.from_workload(w, precisions=(fem.FE_F32_COMP,))
    J, _ = gm.energy_gradient(_dev(w.v))
    assert gm.sync_status() == fem.FE_EDOMAIN
    assert J.item() == math.inf
