"""Failure detection on the device without a fault: the bulk-copy kernels wait for each copy
a bounded number of SM clocks, then give up, record FE_ETIMEOUT, wait for the copies still in
flight and return.  A limit of a few clocks makes that path run on purpose (nothing on the
device is broken: the copies complete, only the wait stops early); the context stays usable
and the next call with the default limit matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, check_grad, energy_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [0, 2], ids=["f64", "df64"])
def test_short_wait_limit_reports_timeout_then_recovers(precision):
    from paper_2109_01158_gb300 import fem
    w = mg.neohooke_cube3d(24)
    gm = fem.FEMesh.from_workload(w, precisions=(precision,))
    v = torch.from_numpy(w.v).cuda()
    gm.set_wait_limit(4)                        # the patch gather's first wait gives up
    gm.energy_gradient(v)
    with pytest.raises(fem.FEError) as err:
        gm.sync_status()
    assert err.value.status == fem.FE_ETIMEOUT
    assert gm.sync_status() == fem.FE_OK        # the status word was cleared
    gm.set_wait_limit(0)                        # default limit: the next call is correct
    J, g = gm.energy_gradient(v)
    assert gm.sync_status() == fem.FE_OK
    om = oracle.OracleMesh(w)
    check_energy(J.item(), om.energy(w.v)[0], energy_scale(om, w.v))
    check_grad(g.cpu().numpy(), om.gradient_exact(w.v)[0])


def test_wait_limit_rejects_negative():
    from paper_2109_01158_gb300 import fem
    w = mg.plaplace_square(4)
    gm = fem.FEMesh.from_workload(w)
    with pytest.raises(fem.FEError):
        gm.set_wait_limit(-1)
