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
def test_batch_in_page_locked_host_memory_with_completion_flags():
    """v, J and g in page-locked host memory (read and written by the kernel directly) give
    bitwise the results of device buffers; each request's completion flag is raised (1);
    the whole batch is one launch."""
    fem, serve = _gpu()
    cat = serve.Catalogue(0)
    keys = [("nh3", 11), ("plap", 3.0, 45), ("nh2", 32), ("plap", 1.5, 23)]
    batch = fem.Batch(0)
    dev_items, host_items = [], []
    for k, key in enumerate(keys):
        mesh = cat.get(key)
        v = serve.request_vector(cat.workloads[key], k)
        dev_items.append(_item(fem, mesh, v))
        it = _item(fem, mesh, v)
        vh = torch.from_numpy(v).pin_memory()
        Jh = torch.zeros(1, dtype=torch.float64).pin_memory()
        gh = torch.zeros(mesh.ndof, dtype=torch.float64).pin_memory()
        done = torch.zeros(1, dtype=torch.int32).pin_memory()
        host_items.append((mesh, vh, Jh, gh, it[4], done))
    n0 = batch.launch_count()
    batch.run(dev_items)
    assert batch.sync_status() == fem.FE_OK
    batch.run(host_items)
    assert batch.sync_status() == fem.FE_OK
    assert batch.launch_count() - n0 == 2
    for d, h in zip(dev_items, host_items):
        assert h[5].item() == 1
        assert h[2].item() == d[2].item()
        np.testing.assert_array_equal(h[3].numpy(), d[3].cpu().numpy())


@pytest.mark.gpu
def test_batch_wait_limit_runs_out_then_recovers():
    """With a wait limit of one SM clock the first gather tile of a large request gives up
    waiting for the element tiles still running (FE_ETIMEOUT, completion flag 3); the next
    call with the default limit returns bitwise the results of a fresh executor."""
    fem, serve = _gpu()
    cat = serve.Catalogue(0)
    key = ("nh3", 38)
    mesh = cat.get(key)
    v = serve.request_vector(cat.workloads[key], 0)
    ref = _item(fem, mesh, v)
    fresh = fem.Batch(0)
    fresh.run([ref])
    assert fresh.sync_status() == fem.FE_OK
    batch = fem.Batch(0)
    with pytest.raises(fem.FEError):
        batch.set_wait_limit(-1)
    batch.set_wait_limit(1)
    it = _item(fem, mesh, v)
    done = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch.run([it + (done,)])
    with pytest.raises(fem.FEError) as e:
        batch.sync_status()
    assert e.value.status == fem.FE_ETIMEOUT and done.item() == 3
    batch.set_wait_limit(0)
    it2 = _item(fem, mesh, v)
    done.zero_()
    batch.run([it2 + (done,)])
    assert batch.sync_status() == fem.FE_OK and done.item() == 1
    assert it2[2].item() == ref[2].item()
    np.testing.assert_array_equal(it2[3].cpu().numpy(), ref[3].cpu().numpy())


@pytest.mark.gpu
def test_native_server_completes_small_requests_before_the_large_one_of_their_batch():
    """A batch holding one large request and several small ones: the small ones run first
    (smallest mesh first) and complete on their own flags, before the large one."""
    fem, serve = _gpu()
    cat = serve.Catalogue(0)
    big, smalls = ("nh3", 70), [("plap", 2.0, 23), ("nh2", 23), ("plap", 3.0, 32), ("nh3", 6)]
    keys = [big] + smalls
    bufs = []
    for k, key in enumerate(keys):
        mesh = cat.get(key)
        v = torch.from_numpy(serve.request_vector(cat.workloads[key], k)).pin_memory()
        g = torch.empty(mesh.ndof, dtype=torch.float64).pin_memory()
        bufs.append((mesh, v, np.empty(1), g))
    srv = fem.NativeServer(0, 2 << 30, 64)
    for _ in range(2):   # the second round is timed: everything is warm
        t0 = srv.now() + 0.02
        tickets = [srv.submit(m, v.numpy(), J, g.numpy(), t0) for m, v, J, g in bufs]
        res = [srv.wait(t) for t in tickets]
    assert all(r[0] == fem.FE_OK for r in res)
    assert len({r[2] for r in res}) == 1          # one batch: the same start time
    t_big = res[0][3]
    assert max(r[3] for r in res[1:]) < t_big
    srv.close()


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


@pytest.mark.gpu
@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
@pytest.mark.parametrize("max_batch", [256, 1], ids=["batched", "serial"])
def test_native_server_results_equal_the_batch_call(max_batch, pinned):
    """fe_server (host vectors in, host results out; staged through its pinned buffers, or
    read and written by the kernel straight in page-locked caller buffers) returns bitwise the
    J and g of the batch call on each request alone, whatever the batching, in one launch per
    batch; every request completes after it arrives and after it started."""
    fem, serve = _gpu()
    cat = serve.Catalogue(0)
    keys = [("plap", 3.0, 23), ("nh3", 8), ("nh2", 45), ("plap", 1.5, 32), ("nh3", 8), ("nh2", 23)] * 3
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
    srv = fem.NativeServer(0, 1 << 30, max_batch)
    t0 = srv.now()
    sub = []
    keep = []
    for k, (key, v) in enumerate(reqs):
        mesh = cat.get(key)
        J, g = np.empty(1), np.empty(mesh.ndof)
        if pinned:
            vt = torch.from_numpy(v).pin_memory()
            gt = torch.empty(mesh.ndof, dtype=torch.float64).pin_memory()
            keep.append((vt, gt))
            v, g = vt.numpy(), gt.numpy()
        sub.append((srv.submit(mesh, v, J, g, t0 + 1e-4 * k), J, g))
    for (ticket, J, g), (Ja, ga) in zip(sub, alone):
        st, ta, ts, td = srv.wait(ticket)
        assert st == fem.FE_OK and ta <= ts <= td
        assert J[0] == Ja
        np.testing.assert_array_equal(g, ga)
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["launches"] == stats["batches"]
    if max_batch == 1:
        assert stats["max_batch"] == 1 and stats["batches"] == len(reqs)
    srv.close()


@pytest.mark.gpu
def test_native_server_admission_arrivals_and_domain_errors():
    fem, serve = _gpu()
    w = mg.neohooke_cube3d(6)
    mesh = fem.FEMesh.from_workload(w, precisions=(fem.FE_DF64,))
    need = fem.Batch.work_bytes(mesh) + 16 * mesh.ndof
    # a request larger than the whole budget is refused at submission
    small = fem.NativeServer(0, need // 2, 8)
    with pytest.raises(fem.FEError):
        small.submit(mesh, w.v.copy(), np.empty(1), np.empty(mesh.ndof))
    small.close()
    # a budget of about one request serialises the batches; a future arrival is not started
    # early; an inverted element gives FE_EDOMAIN and J = +Inf for that request only
    srv = fem.NativeServer(0, need + 4096, 64)
    bad = w.coords.ravel().copy()
    bad[3 * 21] += 2.0
    t0 = srv.now()
    outs = []
    for k, v in enumerate([w.v, bad, w.v]):
        J, g = np.empty(1), np.empty(mesh.ndof)
        outs.append((srv.submit(mesh, np.ascontiguousarray(v), J, g, t0 + 0.05 * (k + 1)), J, g))
    res = [srv.wait(t) for t, _, _ in outs]
    assert [r[0] for r in res] == [fem.FE_OK, fem.FE_EDOMAIN, fem.FE_OK]
    for k, (st, ta, ts, td) in enumerate(res):
        assert ts >= ta >= t0 + 0.05 * (k + 1) - 1e-9
    assert outs[1][1][0] == math.inf and np.isfinite(outs[0][1][0]) and outs[0][1][0] == outs[2][1][0]
    assert srv.stats()["max_batch"] == 1
    srv.close()
