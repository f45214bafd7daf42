"""Serving: batched evaluation over many resident meshes and the continuous-batching loop.

GPU tests: each request's J and g are bitwise the same alone and in a mixed batch, agree
with the oracle within the FP64 tolerances, and the real-time server (batched and serial)
returns those same results.  CPU tests: the synthetic request stream."""
import math

import numpy as np
import pytest

import oracle
from paper_2109_01158_gb300 import meshgen as mg
from parity import check_energy, check_grad, energy_scale

torch = pytest.importorskip("torch")


def test_request_mix_and_arrivals():
    from paper_2109_01158_gb300 import serve
    keys = serve.request_keys(512, seed=3)
    kinds = [k[0] for k in keys]
    frac = {c: kinds.count(c) / 512 for c in ("plap", "nh2", "nh3")}
    assert abs(frac["plap"] - 0.5) < 0.07 and abs(frac["nh2"] - 0.3) < 0.07 and abs(frac["nh3"] - 0.2) < 0.07
    assert {k[1] for k in keys if k[0] == "plap"} == {1.5, 2.0, 3.0}
    ne = [2 * k[-1] ** 2 if k[0] != "nh3" else 6 * k[-1] ** 3 for k in keys]
    assert min(ne) >= 500 and max(ne) <= 2.2e6
    t = serve.poisson_arrivals(4096, rate=200.0, seed=3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0 and np.all(gaps > 0)
    assert keys == serve.request_keys(512, seed=3)


def _gpu():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01158_gb300 import fem, serve
    return fem, serve


def _item(fem, mesh, v):
    dev = torch.device("cuda", 0)
    wb = fem.Batch.work_bytes(mesh)
    work = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
    off = (-work.data_ptr()) % 256
    work = work[off: off + wb]
    J = torch.empty((), dtype=torch.float64, device=dev)
    g = torch.empty(mesh.ndof, dtype=torch.float64, device=dev)
    return (mesh, torch.from_numpy(v).to(dev), J, g, work)


@pytest.mark.gpu
def test_batch_results_same_alone_and_in_the_mix():
    fem, serve = _gpu()
    cat = serve.Catalogue(0)
    keys = [("plap", 3.0, 23), ("plap", 1.5, 32), ("nh2", 45), ("nh3", 8), ("nh2", 23), ("nh3", 11),
            ("plap", 2.0, 64), ("nh3", 8)]
    reqs = []
    for k, key in enumerate(keys):
        cat.get(key)
        reqs.append((key, serve.request_vector(cat.workloads[key], k)))
    batch = fem.Batch(0)
    alone = []
    for key, v in reqs:
        it = _item(fem, cat.get(key), v)
        batch.run([it])
        assert batch.sync_status() == fem.FE_OK
        alone.append((it[2].item(), it[3].cpu().numpy()))
    items = [_item(fem, cat.get(key), v) for key, v in reqs]
    batch.run(items)
    assert batch.sync_status() == fem.FE_OK
    for (Ja, ga), it in zip(alone, items):
        assert it[2].item() == Ja
        np.testing.assert_array_equal(it[3].cpu().numpy(), ga)
    # and against the oracle
    for (key, v), (Ja, ga) in zip(reqs, alone):
        w = cat.workloads[key]
        om = oracle.OracleMesh(w)
        check_energy(Ja, om.energy(v)[0], energy_scale(om, v))
        check_grad(ga, om.gradient_exact(v)[0])


@pytest.mark.gpu
def test_batch_reports_domain_error_per_item():
    fem, serve = _gpu()
    w = mg.neohooke_cube3d(3)
    mesh = fem.FEMesh.from_workload(w, precisions=(fem.FE_DF64,))
    bad = w.coords.ravel().copy()
    bad[3 * 21] += 2.0
    batch = fem.Batch(0)
    good_item, bad_item = _item(fem, mesh, w.v), _item(fem, mesh, bad)
    batch.run([good_item, bad_item])
    assert batch.sync_status() == fem.FE_EDOMAIN
    assert math.isfinite(good_item[2].item()) and bad_item[2].item() == math.inf


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batched", "serial"])
def test_server_stream_results(mode):
    fem, serve = _gpu()
    cat = serve.Catalogue(0)
    reqs = [r for r in serve.make_requests(40, seed=5, rate=2000.0, catalogue=cat)]
    # keep the test quick: cap sizes by replacing large keys
    small = [r for r in reqs if r.ne <= 300000]
    for k, r in enumerate(small):
        r.arrival = k * 2e-4
    server = serve.Server(cat, hbm_budget=1 << 30)
    st = server.run(small, mode=mode)
    assert st.n == len(small) and st.p99_ms >= st.p50_ms > 0
    if mode == "serial":
        assert st.max_batch == 1 and st.steps == len(small)
    batch = fem.Batch(0)
    for r in small[:10]:
        it = _item(fem, cat.get(r.key), r.v)
        batch.run([it])
        batch.sync_status()
        assert it[2].item() == r.J
        np.testing.assert_array_equal(it[3].cpu().numpy(), r.g)
