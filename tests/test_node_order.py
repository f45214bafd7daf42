"""Host-side node renumbering (fe_node_order): the permutations fe_mesh_upload applies for
FE_ORDER_MORTON and FE_ORDER_RCM.  Runs on CPU: fe_node_order does no device work.

Reverse Cuthill-McKee (Cuthill & McKee 1969, reversed by George 1971) is pinned by
properties that fix it independently of the implementation: the optimal bandwidth on a
strip, a bandwidth no worse than scipy's own RCM on shuffled grids, the breadth-first level
structure of the (unreversed) Cuthill-McKee sequence, and contiguous components."""
import numpy as np
import pytest

from paper_2109_01158_gb300 import fem
from paper_2109_01158_gb300 import meshgen as mg


def _shuffled(X, E, seed=0):
    X = np.asarray(X)
    E = np.asarray(E)
    s = np.random.default_rng(seed).permutation(X.shape[0])  # s[new] = old
    inv = np.argsort(s)
    return X[s], inv[E].astype(np.int32)


def _bandwidth(E, perm=None):
    E = np.asarray(E)
    nn = int(E.max()) + 1
    inv = np.arange(nn) if perm is None else np.argsort(perm)
    Ei = inv[E]
    k = E.shape[1]
    return max(int(np.abs(Ei[:, a] - Ei[:, b]).max()) for a in range(k) for b in range(k) if a != b)


def _adjacency(E, nn):
    adj = [set() for _ in range(nn)]
    for el in np.asarray(E):
        for a in el:
            for b in el:
                if a != b:
                    adj[a].add(int(b))
    return adj


def _meshes():
    X, E, _ = mg.lshape_tri(2)
    return [mg.rect_tri(7, 5)[:2], mg.box_tet(3, 4, 2)[:2], (X, E)]


@pytest.mark.parametrize("order", [fem.FE_ORDER_NONE, fem.FE_ORDER_MORTON, fem.FE_ORDER_RCM])
def test_orders_are_permutations(order):
    for X, E in _meshes():
        Xs, Es = _shuffled(X, E)
        p = fem.node_order(Xs, Es, order)
        assert p.dtype == np.int32
        assert np.array_equal(np.sort(p), np.arange(Xs.shape[0]))
        if order == fem.FE_ORDER_NONE:
            assert np.array_equal(p, np.arange(Xs.shape[0]))
        assert np.array_equal(p, fem.node_order(Xs, Es, order))  # deterministic


def test_rcm_strip_reaches_the_optimal_bandwidth():
    """A strip of n squares, each cut into two triangles: 2(n+1) nodes.  No numbering has
    bandwidth 1: that allows a node only the neighbours i - 1 and i + 1, and the strip's
    interior nodes have four.  RCM finds bandwidth 2 from any starting numbering."""
    X, E = mg.rect_tri(30, 1)[:2]
    for seed in range(3):
        Xs, Es = _shuffled(X, E, seed)
        assert _bandwidth(Es) > 20
        assert _bandwidth(Es, fem.node_order(Xs, Es, fem.FE_ORDER_RCM)) == 2


@pytest.mark.parametrize("mesh", ["tri", "tet"])
def test_rcm_bandwidth_matches_scipy(mesh):
    """On shuffled structured meshes the bandwidth is no worse than that of scipy's reverse
    Cuthill-McKee (one more allowed: the two differ in the choice of start node) and near
    the natural numbering's."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    X, E = (mg.rect_tri(40, 25) if mesh == "tri" else mg.box_tet(12, 9, 7))[:2]
    Xs, Es = _shuffled(X, E)
    nn = Xs.shape[0]
    k = Es.shape[1]
    rows = np.repeat(Es, k, axis=1).ravel()
    cols = np.tile(Es, (1, k)).ravel()
    A = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(nn, nn))
    ref = _bandwidth(Es, csgraph.reverse_cuthill_mckee(A, symmetric_mode=True))
    got = _bandwidth(Es, fem.node_order(Xs, Es, fem.FE_ORDER_RCM))
    assert got <= ref + 1
    assert got <= _bandwidth(E)
    assert _bandwidth(Es) > 10 * got


def test_cuthill_mckee_level_structure_and_components():
    """Reversed, the RCM sequence is a Cuthill-McKee sequence.  Every component occupies a
    contiguous range, breadth-first from its first node.  Each later node's earliest-numbered
    neighbour (its parent) sits at a non-decreasing position.  Nodes with the same parent
    come in increasing (degree, id) order.  The mesh is two disjoint grids plus two isolated
    nodes: four components."""
    X1, E1 = mg.rect_tri(6, 4)[:2]
    X2, E2 = mg.rect_tri(3, 5, x0=5.0)[:2]
    n1 = np.asarray(X1).shape[0]
    X = np.vstack([np.asarray(X1), np.full((2, 2), 9.0), np.asarray(X2)])
    E = np.vstack([np.asarray(E1), np.asarray(E2) + n1 + 2]).astype(np.int32)
    Xs, Es = _shuffled(X, E, seed=3)
    nn = Xs.shape[0]
    cm = fem.node_order(Xs, Es, fem.FE_ORDER_RCM)[::-1]
    adj = _adjacency(Es, nn)
    pos = np.empty(nn, dtype=np.int64)
    pos[cm] = np.arange(nn)
    i = 0
    n_comp = 0
    while i < nn:
        root = int(cm[i])
        dist = {root: 0}
        frontier = [root]
        while frontier:
            nxt = []
            for u in frontier:
                for w in sorted(adj[u]):
                    if w not in dist:
                        dist[w] = dist[u] + 1
                        nxt.append(w)
            frontier = nxt
        comp = [int(c) for c in cm[i:i + len(dist)]]
        assert set(comp) == set(dist)                              # contiguous component
        d = [dist[c] for c in comp]
        assert all(a <= b for a, b in zip(d, d[1:]))                # level by level
        parent = [min(pos[w] for w in adj[c]) for c in comp[1:]]
        assert all(a <= b for a, b in zip(parent, parent[1:]))      # FIFO order of parents
        for a, b, pa, pb in zip(comp[1:], comp[2:], parent, parent[1:]):
            if pa == pb:
                assert (len(adj[a]), a) < (len(adj[b]), b)           # siblings by degree, id
        i += len(dist)
        n_comp += 1
    assert n_comp == 4


def test_morton_follows_space_on_an_elongated_domain():
    """Morton keys quantise every axis on the largest extent, so on a 60 x 2 strip of unit
    squares the numbering stays local: a bandwidth at least 4 times below the row-by-row
    numbering's 62 (the Z-curve jumps only at the edges of its power-of-two blocks).
    Quantising each axis on its own extent would order the three rows one after another,
    like the row-by-row numbering."""
    X, E = mg.rect_tri(60, 2, lx=60.0, ly=2.0)[:2]
    Xs, Es = _shuffled(X, E, seed=5)
    got = _bandwidth(Es, fem.node_order(Xs, Es, fem.FE_ORDER_MORTON))
    assert _bandwidth(E) == 62 and 4 * got < 62


def test_node_order_rejects_bad_input():
    X, E = mg.rect_tri(3, 2)[:2]
    with pytest.raises(fem.FEError, match="FE_EINVAL"):
        fem.node_order(X, E, 7)
    bad = np.array(E, dtype=np.int32)
    bad[0, 0] = X.shape[0]
    with pytest.raises(fem.FEError, match="out of range"):
        fem.node_order(X, bad, fem.FE_ORDER_RCM)


def test_size_limits_and_empty_meshes():
    """The size checks fe_mesh_upload shares with fe_node_order reject n_nodes >= 2^31 and
    n_elems*(dim+1) >= 2^31 before reading any array; an empty mesh is accepted, and nodes
    that belong to no element are still numbered (each is its own component)."""
    lib = fem.load_library()   # argument types set by the binding
    X = np.zeros((4, 3))
    E = np.zeros((1, 4), dtype=np.int32)
    perm = np.empty(4, dtype=np.int32)
    call = lib.fe_node_order
    assert call(3, 1 << 31, X.ctypes.data, 0, None, fem.FE_ORDER_RCM, perm.ctypes.data) == fem.FE_EINVAL
    assert "too large" in fem.fe_last_error()
    assert call(3, 4, X.ctypes.data, 1 << 29, E.ctypes.data, fem.FE_ORDER_RCM, perm.ctypes.data) == fem.FE_EINVAL
    assert call(3, 0, None, 0, None, fem.FE_ORDER_RCM, None) == fem.FE_OK
    for order in (fem.FE_ORDER_MORTON, fem.FE_ORDER_RCM):
        p = fem.node_order(np.random.default_rng(1).random((7, 2)), np.zeros((0, 3), np.int32), order)
        assert np.array_equal(np.sort(p), np.arange(7))
