"""The device L-BFGS memory (fe_lbfgs, compact representation) against the two-loop
recursion in torch on the same pairs, through the ring of pairs (fewer than m, exactly m,
wrapped around), a rejected pair and a reset; and L-BFGS minimisations driven by it."""
import numpy as np
import pytest

from paper_2109_01158_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _fem():
    from paper_2109_01158_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01158_gb300 import fem
    return fem


def _pairs(n, count, seed):
    """count pairs of a strictly convex quadratic with a spread spectrum: y = A s."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    diag = torch.exp(torch.linspace(0.0, 6.0, n, dtype=torch.float64))
    out = []
    v = torch.randn(n, generator=gen, dtype=torch.float64)
    for _ in range(count):
        v_new = v + torch.randn(n, generator=gen, dtype=torch.float64) * 0.1
        out.append((v_new.cuda(), v.cuda(), (diag * v_new).cuda(), (diag * v).cuda()))
        v = v_new
    return out


@pytest.mark.parametrize("count", [0, 1, 3, 10, 17])
def test_device_direction_matches_two_loop(count):
    fem = _fem()
    from paper_2109_01158_gb300.minimize import _State
    n, m = 4099, 10
    mem = fem.LbfgsMemory(n, m)
    g0 = torch.randn(n, dtype=torch.float64, generator=torch.Generator().manual_seed(99)).cuda()
    ref = _State(torch.zeros(n, dtype=torch.float64, device="cuda"), 0.0, g0, m)
    for v_new, v, g_new, g in _pairs(n, count, seed=count):
        sy = mem.update(v_new, v, g_new, g)
        assert sy > 0.0
        ref.g = g
        ref.v = v
        ref.accept(v_new, 0.0, g_new)
    assert mem.pairs() == min(count, m)
    ref.g = g0
    d_ref, gd_ref = ref.direction()
    d, gd = mem.direction(g0)
    scale = float(d_ref.abs().max())
    assert float((d - d_ref).abs().max()) <= 1e-11 * scale
    assert abs(gd - gd_ref) <= 1e-11 * abs(gd_ref) and gd < 0.0
    d2, gd2 = mem.direction(g0)
    assert torch.equal(d, d2) and gd == gd2
    mem.close()


def test_rejected_pair_and_reset():
    fem = _fem()
    n = 1000
    mem = fem.LbfgsMemory(n, 4)
    (v_new, v, g_new, g), = _pairs(n, 1, seed=5)
    assert mem.update(v_new, v, g_new, g) > 0.0 and mem.pairs() == 1
    assert mem.update(v_new, v, g, g_new) < 0.0 and mem.pairs() == 1     # s.y < 0: not kept
    mem.reset()
    assert mem.pairs() == 0
    d, gd = mem.direction(g)
    torch.testing.assert_close(d, -g / g.norm(), rtol=1e-15, atol=0.0)
    assert abs(gd + float(g.norm())) <= 1e-14 * float(g.norm())
    with pytest.raises(fem.FEError):
        fem.LbfgsMemory(n, 17)
    mem.close()


def test_lbfgs_with_device_memory_reaches_the_same_minimum():
    fem = _fem()
    from paper_2109_01158_gb300 import minimize
    w = mg.neohooke_cube3d(12)
    w.f = np.tile([0.0, 0.0, -1e-2], w.nn)
    gm = fem.FEMesh.from_workload(w)
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    u0 = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    ref = minimize.lbfgs(minimize.mesh_evaluator(gm), u0, gtol=1e-8, relative=True)
    dev = minimize.lbfgs(minimize.mesh_evaluator(gm), u0, gtol=1e-8, relative=True, device_memory=True)
    again = minimize.lbfgs(minimize.mesh_evaluator(gm), u0, gtol=1e-8, relative=True, device_memory=True)
    assert ref.converged and dev.converged
    assert abs(dev.J - ref.J) <= 1e-13 * abs(ref.J)
    assert dev.iters <= 1.2 * ref.iters + 5
    assert again.J == dev.J and again.iters == dev.iters and torch.equal(again.v, dev.v)


def test_step_equals_update_then_direction():
    """fe_lbfgs_step gives bitwise the pairs and directions of update + direction, and drops a
    pair with s.y <= 0 (the direction then comes from the pairs kept before)."""
    fem = _fem()
    n, m = 3001, 4
    a, b = fem.LbfgsMemory(n, m), fem.LbfgsMemory(n, m)
    for v_new, v, g_new, g in _pairs(n, 7, seed=11):
        a.update(v_new, v, g_new, g)
        da, gda = a.direction(g_new)
        db, sy, gdb, gmax = b.step(v_new, v, g_new, g)
        assert sy > 0.0 and a.pairs() == b.pairs()
        assert torch.equal(da, db) and gda == gdb
        assert gmax == float(g_new.abs().max())
    # a pair with s.y < 0 is not kept
    k = b.pairs()
    db, sy, gdb, _ = b.step(v, v_new, g_new, g)
    assert sy < 0.0 and b.pairs() == k
    da, gda = a.direction(g_new)
    assert torch.equal(da, db) and gda == gdb
    a.close()
    b.close()


def test_smallest_memory_and_one_unknown():
    """n = 1 and m = 1: on f(x) = a x^2 / 2 the memory holds the exact curvature, so the
    direction from any gradient is the Newton step -g / a; a second pair replaces the first."""
    fem = _fem()
    mem = fem.LbfgsMemory(1, 1)
    a = 3.0
    x0, x1, x2 = (torch.tensor([t], dtype=torch.float64, device="cuda") for t in (1.0, 0.5, 0.25))
    assert mem.update(x1, x0, a * x1, a * x0) > 0.0 and mem.pairs() == 1
    assert mem.update(x2, x1, a * x2, a * x1) > 0.0 and mem.pairs() == 1
    g = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    d, gd = mem.direction(g)
    assert abs(float(d[0]) + 0.7 / a) <= 1e-15 and abs(gd + 0.49 / a) <= 1e-15
    mem.close()


def test_memory_save_restore_gives_bitwise_directions():
    """fe_lbfgs_save / fe_lbfgs_restore: a memory restored from a saved one (wrapped ring, so
    the pairs sit in other slots) gives bitwise the same directions and, after one more pair,
    the same updates; restoring more pairs than m is refused."""
    fem = _fem()
    n, m = 3001, 5
    a = fem.LbfgsMemory(n, m)
    for v_new, v, g_new, g in _pairs(n, 8, seed=5):    # 8 > m: the ring has wrapped
        a.update(v_new, v, g_new, g)
    state = a.save()
    assert state[0].shape == (m, n) and state[2].shape == (m, m)
    b = fem.LbfgsMemory(n, m)
    b.restore(state)
    assert b.pairs() == m
    g0 = torch.randn(n, dtype=torch.float64, generator=torch.Generator().manual_seed(3)).cuda()
    da, gda = a.direction(g0)
    db, gdb = b.direction(g0)
    assert torch.equal(da, db) and gda == gdb
    (v_new, v, g_new, g), = _pairs(n, 1, seed=11)
    assert a.update(v_new, v, g_new, g) == b.update(v_new, v, g_new, g)
    da, _ = a.direction(g0)
    db, _ = b.direction(g0)
    assert torch.equal(da, db)
    small = fem.LbfgsMemory(n, m - 1)
    with pytest.raises(fem.FEError):
        small.restore(state)
    empty = fem.LbfgsMemory(n, m)
    empty.restore(fem.LbfgsMemory(n, m).save())
    assert empty.pairs() == 0
    for x in (a, b, small, empty):
        x.close()


@pytest.mark.parametrize("precision", ["f64", "df64"])
def test_lbfgs_checkpoint_and_resume_continue_bitwise(precision):
    """An L-BFGS run stopped at 25 iterations with a checkpoint, the checkpoint pickled and
    resumed, reaches bitwise the iterate, J, counters and history of one uninterrupted run."""
    import pickle
    fem = _fem()
    from paper_2109_01158_gb300 import minimize
    w = mg.neohooke_cube3d(10)
    w.f = np.tile([0.0, 0.0, -1e-2], w.nn)
    prec = fem.FE_F64 if precision == "f64" else fem.FE_DF64
    gm = fem.FEMesh.from_workload(w, precisions=(prec,))
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    u0 = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    kw = dict(gtol=1e-9, relative=True, device_memory=True)
    full = minimize.lbfgs(minimize.mesh_evaluator(gm), u0, max_iter=60, **kw)
    part = minimize.lbfgs(minimize.mesh_evaluator(gm), u0, max_iter=25, checkpoint=True, **kw)
    assert part.iters == 25 and part.checkpoint is not None
    ck = pickle.loads(pickle.dumps(part.checkpoint))
    rest = minimize.lbfgs(minimize.mesh_evaluator(gm), u0, max_iter=60, resume=ck, **kw)
    assert rest.iters == full.iters and rest.evals == full.evals
    assert rest.J == full.J and torch.equal(rest.v, full.v)
    assert rest.history == full.history
    with pytest.raises(ValueError):
        minimize.lbfgs(minimize.mesh_evaluator(gm), u0, max_iter=60, resume=ck, gtol=1e-9, relative=True)
