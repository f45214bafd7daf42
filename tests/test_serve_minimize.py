"""Continuous batching of whole minimisations (serve.MinimizeServer): requests arriving over
time are admitted by arrival and device bytes, their L-BFGS trial points are evaluated
together in one batched launch per round, and every result equals the result of the same
request served alone (the one-at-a-time mode) bit for bit."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _serve():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01158_gb300 import serve
    return serve


def test_served_minimisations_equal_alone_and_in_the_mix():
    serve = _serve()
    kw = dict(n=6, sizes=(4, 6, 8), rate=400.0, gtol=1e-8)
    mixed, alone = serve.make_minimize_requests(**kw), serve.make_minimize_requests(**kw)
    srv = serve.MinimizeServer(0)
    sb = srv.run(mixed, "batched")
    ss = srv.run(alone, "serial")
    srv.close()
    assert sb.max_active > 1 and ss.max_active == 1
    assert sb.evaluations == ss.evaluations and sb.rounds < ss.rounds
    for a, b in zip(mixed, alone):
        assert a.result.converged and b.result.converged
        assert a.result.J == b.result.J and a.result.iters == b.result.iters
        assert torch.equal(a.result.v, b.result.v)
        assert a.t_admit >= a.arrival - 1e-9 and a.t_done > a.t_admit


def test_minimisations_are_admitted_within_the_hbm_budget():
    serve = _serve()
    reqs = serve.make_minimize_requests(n=6, sizes=(6, 8), rate=1e6, gtol=1e-6)
    srv = serve.MinimizeServer(0)
    smallest = min(srv.job_bytes(r.mesh) for r in reqs)
    largest = max(srv.job_bytes(r.mesh) for r in reqs)
    srv.budget = 2 * largest
    st = srv.run(reqs, "batched")
    srv.close()
    assert 2 <= st.max_active <= (2 * largest) // smallest
    assert all(r.result.converged for r in reqs)
