"""fe_energy_noalloc: the energy entry point for callers that cannot let this library
allocate device memory (their GPU memory belongs to their own allocator, or their loop must
not call cudaMalloc).  Called through the C ABI and checked against fe_energy, the regular
entry point, and against the oracle, within the energy tolerance of the other parity tests,
on two calls in a row (the second call reuses the static scratch the first one left behind).
Also: small strains against a 50-digit reference (the density is evaluated in displacement
form, as in the context kernels), no load, an empty mesh, an inverted element (+Inf), a node
id outside the mesh (NaN, nothing read through it) and the arguments it rejects.

This file is collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, energy_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


class _Args:
    """Device copies of one workload in the layouts fe_energy_noalloc takes; dphi, vol and b
    come from the oracle's precompute (the caller computes them)."""

    def __init__(self, w):
        self.w = w
        self.om = oracle.OracleMesh(w)
        self.coords = _dev(w.coords.ravel(), np.float64)
        self.elems = _dev(w.elems.ravel(), np.int32)
        self.dphi = _dev(self.om.dphi, np.float64)
        self.vol = _dev(self.om.vol, np.float64)
        self.b = _dev(self.om.b, np.float64) if w.f is not None else None
        self.v = _dev(w.v, np.float64)
        self.J = torch.empty((), dtype=torch.float64, device="cuda")

    def call(self, model=None, ne=None, b=True):
        from paper_2109_01158_gb300 import fem
        w = self.w
        self.J.fill_(-12345.0)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        bp = self.b.data_ptr() if (b and self.b is not None) else None
        fem.fe_energy_noalloc(0, stream, w.dim, w.d, w.model if model is None else model, float(w.p),
                              float(w.C1), float(w.D1), w.nn, self.coords.data_ptr(),
                              w.ne if ne is None else ne, self.elems.data_ptr(), self.dphi.data_ptr(),
                              self.vol.data_ptr(), bp, self.v.data_ptr(), self.J.data_ptr())
        torch.cuda.synchronize()
        return self.J.item()


def _lshape_lp(level=3):
    coords, elems, bnd = mg.lshape_tri(level)
    v = mg.uniform(7, np.arange(coords.shape[0]), -1.0, 1.0) * (1 - bnd)
    return mg.Workload(f"lshape{level}", 2, 1, coords, elems, bnd.astype(np.uint8), mg.MODEL_PLAPLACE_LP,
                       p=3.0, f=np.full(coords.shape[0], -10.0), v=v)


@pytest.mark.parametrize("maker", [
    lambda: mg.neohooke_cube3d(20),
    lambda: mg.neohooke_rect2d(96, 48),
    lambda: mg.plaplace_square(40),
    lambda: mg.random_small(5, 3, mg.MODEL_PLAPLACE, 7, 6, 5, p=1.5),
    _lshape_lp,
], ids=["nh3d", "nh2d", "plap2d", "plap3d_p1.5", "lshape_lp"])
def test_noalloc_energy_matches_fe_energy_and_oracle_on_two_calls(maker):
    from paper_2109_01158_gb300 import fem
    w = maker()
    gm = fem.FEMesh.from_workload(w)
    J_ref = gm.energy(_dev(w.v)).item()               # the regular entry point
    assert gm.sync_status() == fem.FE_OK
    a = _Args(w)
    J_or, st = a.om.energy(w.v)
    assert st == oracle.OK
    scale = energy_scale(a.om, w.v)
    for _ in range(2):
        J = a.call()
        check_energy(J, J_ref, scale)
        err = check_energy(J, J_or, scale)
    print(f"{w.name}: |J - J_oracle| / scale = {err:.2e}")


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_noalloc_small_strain_homogeneous_energy(eps):
    """v = (I + eps B) X on the unit cube: J = W(I + eps B) exactly (50-digit reference).  The
    formula as written would lose about 1e-16 / eps^2 relative; the displacement form keeps
    the rounding of the input itself, about 4.4e-16 / eps relative (v = X + u in FP64)."""
    from decimal import Decimal, getcontext
    w = mg.neohooke_cube3d(6)
    w.dirichlet[:] = 0
    w.f = None
    B = np.array([[0.3, -0.2, 0.1], [0.05, -0.4, 0.2], [-0.1, 0.25, 0.15]])
    A = np.eye(3) + eps * B
    w.v = (w.coords @ A.T).ravel()
    getcontext().prec = 50
    a50 = [[Decimal(repr(float(x))) for x in row] for row in A]
    det = (a50[0][0] * (a50[1][1] * a50[2][2] - a50[1][2] * a50[2][1])
           - a50[0][1] * (a50[1][0] * a50[2][2] - a50[1][2] * a50[2][0])
           + a50[0][2] * (a50[1][0] * a50[2][1] - a50[1][1] * a50[2][0]))
    I1 = sum(x * x for row in a50 for x in row)
    ref = float(Decimal(repr(w.C1)) * (I1 - 3 - 2 * det.ln()) + Decimal(repr(w.D1)) * (det - 1) ** 2)
    J = _Args(w).call()
    assert abs(J - ref) <= (1e-12 + 4.4e-16 / eps) * abs(ref), (J, ref, abs(J - ref) / abs(ref))


def test_noalloc_without_load_and_empty_mesh():
    """b_dev = NULL is the zero load (same J as fe_energy on the mesh without a load); an
    empty element range gives J = -b.v, and 0 without a load."""
    from paper_2109_01158_gb300 import fem
    w = mg.neohooke_rect2d(40, 20)
    w.f = None
    a = _Args(w)
    gm = fem.FEMesh.from_workload(w)
    check_energy(a.call(b=False), gm.energy(_dev(w.v)).item(), energy_scale(a.om, w.v))
    assert a.call(ne=0, b=False) == 0.0
    w2 = mg.plaplace_square(16)
    a2 = _Args(w2)
    bv = float(np.dot(a2.om.b, w2.v))
    J0 = a2.call(ne=0)
    assert abs(J0 + bv) <= 1e-13 * max(1.0, float(np.abs(a2.om.b * w2.v).sum())), (J0, -bv)


def test_noalloc_inverted_element_gives_inf_then_recovers():
    """One element with det F <= 0 makes J = +Inf; the next call on a valid v is finite and
    correct (the flag word does not carry over)."""
    w = mg.neohooke_cube3d(6)
    a = _Args(w)
    good = a.call()
    vbad = w.v.reshape(-1, 3).copy()
    n0, n1 = int(w.elems[0, 0]), int(w.elems[0, 1])
    vbad[n1], vbad[n0] = w.v.reshape(-1, 3)[n0], w.v.reshape(-1, 3)[n1]   # swap two vertices
    a.v = _dev(vbad.ravel(), np.float64)
    assert a.call() == math.inf
    a.v = _dev(w.v, np.float64)
    check_energy(a.call(), good, energy_scale(a.om, w.v))


def test_noalloc_node_id_outside_the_mesh_gives_nan_then_recovers():
    """An element naming node n_nodes is skipped without reading through it and J = NaN;
    the next call on valid ids gives the right J."""
    w = mg.plaplace_square(12)
    a = _Args(w)
    good = a.call()
    bad = w.elems.copy()
    bad[3, 1] = w.nn
    a.elems = _dev(bad.ravel(), np.int32)
    assert math.isnan(a.call())
    bad[3, 1] = -1
    a.elems = _dev(bad.ravel(), np.int32)
    assert math.isnan(a.call())
    a.elems = _dev(w.elems.ravel(), np.int32)
    check_energy(a.call(), good, energy_scale(a.om, w.v))


def test_noalloc_rejects_bad_arguments():
    from paper_2109_01158_gb300 import fem
    J_d = torch.zeros((), dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")

    def call(model=fem.FE_NEOHOOKE, dim=3, d=3, ne=1, device=0):
        fem.fe_energy_noalloc(device, None, dim, d, model, 2.0, 1.0, 1.0, 2, x.data_ptr(), ne, x.data_ptr(),
                              x.data_ptr(), x.data_ptr(), None, x.data_ptr(), J_d.data_ptr())

    with pytest.raises(fem.FEError) as err:
        call(ne=1 << 30)
    assert err.value.status == fem.FE_EINVAL and "maximum" in str(err.value)
    with pytest.raises(fem.FEError) as err:
        call(model=7)
    assert err.value.status == fem.FE_EINVAL and "unknown model" in str(err.value)
    with pytest.raises(fem.FEError) as err:
        call(model=fem.FE_PLAPLACE_LP, d=3)
    assert err.value.status == fem.FE_EINVAL and "do not match" in str(err.value)
    with pytest.raises(fem.FEError) as err:
        call(device=torch.cuda.device_count())
    assert err.value.status == fem.FE_EINVAL and "no such device" in str(err.value)
