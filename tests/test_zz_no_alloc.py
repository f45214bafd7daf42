"""fe_energy_noalloc: the energy entry point for callers that cannot let this library
allocate device memory (their GPU memory belongs to their own allocator, or their loop must
not call cudaMalloc).  Called through the C ABI and checked against fe_energy, the regular
entry point, within the energy tolerance of the other parity tests, on two calls in a row
(the second call reuses the static scratch the first one left behind).

This file is collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

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


@pytest.mark.parametrize("maker", [
    lambda: mg.neohooke_cube3d(20),
    lambda: mg.neohooke_rect2d(96, 48),
    lambda: mg.plaplace_square(40),
])
def test_noalloc_energy_matches_fe_energy_on_two_calls(maker):
    from paper_2109_01158_gb300 import fem
    w = maker()
    gm = fem.FEMesh.from_workload(w)
    v = _dev(w.v)
    J_ref = gm.energy(v).item()                       # the regular entry point
    assert gm.sync_status() == fem.FE_OK
    dphi, vol = gm.shape_gradients()
    b = gm.load_vector()
    coords_d = _dev(w.coords.ravel(), np.float64)
    elems_d = _dev(w.elems.ravel(), np.int32)
    dphi_d, vol_d, b_d = _dev(dphi), _dev(vol), _dev(b)
    J_d = torch.empty((), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    scale = energy_scale(oracle.OracleMesh(w), w.v)
    for _ in range(2):
        J_d.fill_(float("nan"))
        fem.fe_energy_noalloc(0, stream, w.dim, w.d, w.model, float(w.p), float(w.C1), float(w.D1),
                              w.nn, coords_d.data_ptr(), w.ne, elems_d.data_ptr(), dphi_d.data_ptr(),
                              vol_d.data_ptr(), b_d.data_ptr(), v.data_ptr(), J_d.data_ptr())
        torch.cuda.synchronize()
        check_energy(J_d.item(), J_ref, scale)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_2109_01158_gb300 import fem
    J_d = torch.zeros((), dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(fem.FEError) as err:
        fem.fe_energy_noalloc(0, None, 3, 3, fem.FE_NEOHOOKE, 2.0, 1.0, 1.0, 8, x.data_ptr(),
                              1 << 30, x.data_ptr(), x.data_ptr(), x.data_ptr(), None, x.data_ptr(),
                              J_d.data_ptr())
    assert err.value.status == fem.FE_EINVAL and "maximum" in str(err.value)
