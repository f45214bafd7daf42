"""Seeded synthetic inputs: structured P1 meshes, Dirichlet masks, trial vectors, loads.

This module holds no arithmetic of the method itself (no shape-function gradients,
no volumes, no densities, no mass matrix).  It only produces the *inputs* that the
energy evaluation consumes, in the layout of the paper's ``mesh`` structure
(Section 4.1): ``elems2nodes`` (ne x (dim+1), 0-based here), ``nodes2coord``
(nn x dim), a Dirichlet mask per degree of freedom, and the trial vector ``v`` in the
paper's interleaved dof order (Section 5, eq. (bvvectors): dof n = d*i + j, 0-based).

Both the CPU oracle and the CUDA path consume exactly these arrays.

Random numbers: a counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  The k-th draw for seed s is
mix(s * G + (k + 1) * G) with G = 0x9E3779B97F4A7C15, mapped to [0,1) with 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: one 64-bit draw per counter value in ``idx``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _G + (idx + np.uint64(1)) * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, idx: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Uniform draws in [lo, hi) from 53-bit SplitMix64 outputs, one per counter."""
    z = splitmix64(seed, idx)
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u01


# ----------------------------------------------------------------------------------
# Structured meshes
# ----------------------------------------------------------------------------------

def rect_tri(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0, x0: float = 0.0, y0: float = 0.0):
    """Rectangle [x0,x0+lx]x[y0,y0+ly] cut into nx*ny squares, each split along the
    diagonal (i,j)-(i+1,j+1) into two counter-clockwise right triangles.

    Node (i,j) has index j*(nx+1)+i.  Returns (coords[nn,2] f64, elems[ne,3] int32).
    """
    xs = x0 + lx * np.arange(nx + 1, dtype=np.float64) / nx
    ys = y0 + ly * np.arange(ny + 1, dtype=np.float64) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    n00 = j * (nx + 1) + i
    n10 = n00 + 1
    n01 = n00 + (nx + 1)
    n11 = n01 + 1
    t1 = np.stack([n00, n10, n11], axis=1)
    t2 = np.stack([n00, n11, n01], axis=1)
    elems = np.empty((2 * nx * ny, 3), dtype=np.int32)
    elems[0::2] = t1
    elems[1::2] = t2
    return coords, elems


# The six Kuhn (Freudenthal) tetrahedra of the unit cube: each walks from corner
# (0,0,0) to (1,1,1) along the axes in the order of one permutation.  Vertex lists are
# written so that every tetrahedron is positively oriented.
_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _kuhn_local():
    tets = []
    for perm in _KUHN_PERMS:
        c = [0, 0, 0]
        path = [tuple(c)]
        for ax in perm:
            c[ax] = 1
            path.append(tuple(c))
        # orientation: sign of the permutation; odd permutations get two vertices swapped
        inv = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        if inv % 2 == 1:
            path[2], path[3] = path[3], path[2]
        tets.append(path)
    return tets


def box_tet(nx: int, ny: int, nz: int, lx=1.0, ly=1.0, lz=1.0, x0=0.0, y0=0.0, z0=0.0):
    """Box cut into nx*ny*nz hexahedra, each into the 6 Kuhn tetrahedra (conforming).

    Node (i,j,k) has index (k*(ny+1)+j)*(nx+1)+i.  Returns (coords[nn,3], elems[ne,4]).
    """
    xs = x0 + lx * np.arange(nx + 1, dtype=np.float64) / nx
    ys = y0 + ly * np.arange(ny + 1, dtype=np.float64) / ny
    zs = z0 + lz * np.arange(nz + 1, dtype=np.float64) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    k = k.ravel()

    def nid(di, dj, dk):
        return ((k + dk) * (ny + 1) + (j + dj)) * (nx + 1) + (i + di)

    local = _kuhn_local()
    nh = nx * ny * nz
    elems = np.empty((6 * nh, 4), dtype=np.int32)
    for t, path in enumerate(local):
        for l, (a, b, c) in enumerate(path):
            elems[t::6, l] = nid(a, b, c)
    return coords, elems


def lshape_tri(level: int):
    """L-shaped domain (-1,1)^2 minus the quadrant (0,1)x(-1,0) on a right-triangle grid
    with 2^(level+2) squares per side of (-1,1)^2.  Level 0 has 24 triangles and 21 nodes
    (the example of Section 3); level 1 has 33 free nodes (Benchmark 6 table).
    Returns (coords, elems, boundary_node_mask)."""
    n = 2 ** (level + 2)            # squares per side of the full (-1,1)^2 box
    coords, elems = rect_tri(n, n, 2.0, 2.0, -1.0, -1.0)
    cx = coords[elems].mean(axis=1)
    keep = ~((cx[:, 0] > 0.0) & (cx[:, 1] < 0.0))
    elems = elems[keep]
    used = np.zeros(coords.shape[0], dtype=bool)
    used[elems.ravel()] = True
    new_id = -np.ones(coords.shape[0], dtype=np.int64)
    new_id[used] = np.arange(int(used.sum()))
    coords = coords[used]
    elems = new_id[elems].astype(np.int32)
    x, y = coords[:, 0], coords[:, 1]
    eps = 1e-12
    bnd = (np.abs(x + 1) < eps) | (np.abs(x - 1) < eps) | (np.abs(y + 1) < eps) | (np.abs(y - 1) < eps)
    bnd |= (np.abs(x) < eps) & (y <= eps)
    bnd |= (np.abs(y) < eps) & (x >= -eps)
    return coords, elems, bnd


# ----------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------

def lame_c1_d1(E: float, nu: float):
    """Material constants of the Neo-Hookean density from Young's modulus and Poisson's
    ratio: C1 = mu/2, D1 = K/2, mu = E/(2(1+nu)), K = E/(3(1-2nu)) (Benchmark 2)."""
    mu = E / (2.0 * (1.0 + nu))
    K = E / (3.0 * (1.0 - 2.0 * nu))
    return mu / 2.0, K / 2.0


MODEL_PLAPLACE = 0
MODEL_NEOHOOKE = 1
MODEL_PLAPLACE_LP = 2   # (1/p) sum_m |dv/dx_m|^p: the l^p-norm reading of |grad v|^p


@dataclass
class Workload:
    """One evaluation problem: mesh, boundary mask, model, load and trial vector."""
    name: str
    dim: int
    d: int
    coords: np.ndarray            # nn x dim, float64
    elems: np.ndarray             # ne x (dim+1), int32, 0-based
    dirichlet: np.ndarray         # nn*d uint8 (1 = fixed dof), interleaved dof order
    model: int
    p: float = 2.0
    C1: float = 0.0
    D1: float = 0.0
    f: np.ndarray | None = None   # nodal load f in V_h, nn*d interleaved (None = 0)
    v: np.ndarray | None = None   # trial vector, nn*d interleaved
    eps: float = 1e-6             # central-difference step used by this workload
    extra: dict = field(default_factory=dict)

    @property
    def nn(self) -> int:
        return int(self.coords.shape[0])

    @property
    def ne(self) -> int:
        return int(self.elems.shape[0])

    @property
    def ndof(self) -> int:
        return self.nn * self.d


def plaplace_square(n: int = 64, p: float = 3.0, f: float = -10.0, seed: int = 0) -> Workload:
    """2D p-Laplacian on the unit square, n x n squares x 2 right triangles, zero
    Dirichlet boundary, v ~ U[-1,1] on free nodes (counter = node index), load f."""
    coords, elems = rect_tri(n, n)
    x, y = coords[:, 0], coords[:, 1]
    tol = 1e-12
    bnd = (x < tol) | (x > 1 - tol) | (y < tol) | (y > 1 - tol)
    v = uniform(seed, np.arange(coords.shape[0]), -1.0, 1.0)
    v[bnd] = 0.0
    return Workload(
        name=f"plaplace2d_p{p:g}_{n}x{n}x2", dim=2, d=1, coords=coords, elems=elems,
        dirichlet=bnd.astype(np.uint8), model=MODEL_PLAPLACE, p=p,
        f=np.full(coords.shape[0], f, dtype=np.float64), v=v, eps=1e-6)


def neohooke_rect2d(nx: int = 1024, ny: int = 512, E: float = 1e4, nu: float = 0.3,
                    seed: int = 1, noise: float = 1e-4) -> Workload:
    """2D compressible Neo-Hookean on [0,2]x[0,1], nx x ny squares x 2 triangles, left
    edge clamped.  Load f = -1750*(1,1) (the paper's 2D load scaled by E/2e8); the
    displacement is u = 0.1*x*dir + U[-noise,noise] with dir = (-1,-1)/sqrt(2), u = 0 on
    the clamped edge, and v = X + u (v is the deformation).

    The default noise is 1e-4 (5% of the spacing h = 1/512): noise of 1e-3 is 51% of h and
    folds 28,819 of the 1,048,576 triangles of the 1024x512 mesh (det F <= 0, J = +Inf)."""
    coords, elems = rect_tri(nx, ny, 2.0, 1.0)
    nn = coords.shape[0]
    clamped = coords[:, 0] < 1e-12
    dirichlet = np.repeat(clamped, 2).astype(np.uint8)
    direc = np.array([-1.0, -1.0]) / math.sqrt(2.0)
    u = 0.1 * coords[:, :1] * direc[None, :]
    u = u.ravel() + uniform(seed, np.arange(2 * nn), -noise, noise)
    u[dirichlet.astype(bool)] = 0.0
    v = coords.ravel() + u
    C1, D1 = lame_c1_d1(E, nu)
    f = np.tile(np.array([-1750.0, -1750.0]), nn)
    return Workload(
        name=f"neohooke2d_{nx}x{ny}x2", dim=2, d=2, coords=coords, elems=elems,
        dirichlet=dirichlet, model=MODEL_NEOHOOKE, C1=C1, D1=D1, f=f, v=v, eps=1e-6)


def neohooke_cube3d(n: int = 128, E: float = 1e4, nu: float = 0.3, seed: int = 2,
                    amp: float = 0.05, noise: float = 1e-4) -> Workload:
    """3D compressible Neo-Hookean on the unit cube, n^3 hexahedra x 6 Kuhn tetrahedra,
    face x=0 clamped, f = 0, u_j = amp*sin(pi x) + U[-noise,noise] per component
    (counter = dof index), u = 0 on the clamped face, v = X + u."""
    coords, elems = box_tet(n, n, n)
    nn = coords.shape[0]
    clamped = coords[:, 0] < 1e-12
    dirichlet = np.repeat(clamped, 3).astype(np.uint8)
    u = np.repeat(amp * np.sin(math.pi * coords[:, 0]), 3)
    u = u + uniform(seed, np.arange(3 * nn), -noise, noise)
    u[dirichlet.astype(bool)] = 0.0
    v = coords.ravel() + u
    C1, D1 = lame_c1_d1(E, nu)
    return Workload(
        name=f"neohooke3d_{n}^3x6", dim=3, d=3, coords=coords, elems=elems,
        dirichlet=dirichlet, model=MODEL_NEOHOOKE, C1=C1, D1=D1, f=None, v=v, eps=1e-6)


def twisted_bar(level: int, alpha: float = 2.0 * math.pi, E: float = 2e8, nu: float = 0.3) -> Workload:
    """Benchmark 2: bar (0,0.4)x(-0.005,0.005)^2 meshed with (80*2^(L-1)) x 2^L x 2^L
    hexahedra x 6 tetrahedra, both end faces fixed, v given by the twisting map of
    eq. (displacement) at every node."""
    lx, ly, lz = 0.4, 0.01, 0.01
    nx, ny, nz = 80 * 2 ** (level - 1), 2 ** level, 2 ** level
    coords, elems = box_tet(nx, ny, nz, lx, ly, lz, 0.0, -ly / 2, -lz / 2)
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    ends = (x < 1e-12) | (x > lx - 1e-12)
    dirichlet = np.repeat(ends, 3).astype(np.uint8)
    a = alpha * x / lx
    v = np.stack([x, np.cos(a) * y + np.sin(a) * z, -np.sin(a) * y + np.cos(a) * z], axis=1).ravel()
    C1, D1 = lame_c1_d1(E, nu)
    return Workload(
        name=f"twisted_bar_L{level}", dim=3, d=3, coords=coords, elems=elems,
        dirichlet=dirichlet, model=MODEL_NEOHOOKE, C1=C1, D1=D1, f=None, v=v, eps=1e-6,
        extra={"lx": lx, "ly": ly, "lz": lz, "alpha": alpha})


def shuffle_nodes(w: Workload, seed: int = 4) -> Workload:
    """Same problem with node ids randomly permuted (counter-based keys, seed)."""
    keys = splitmix64(seed, np.arange(w.nn))
    perm = np.argsort(keys, kind="stable")          # new node k is old node perm[k]
    inv = np.empty_like(perm)
    inv[perm] = np.arange(w.nn)
    d = w.d

    def per_dof(a):
        return None if a is None else a.reshape(w.nn, d)[perm].ravel().copy()

    return Workload(
        name=w.name + "_shuffled", dim=w.dim, d=d, coords=w.coords[perm].copy(),
        elems=inv[w.elems].astype(np.int32), dirichlet=per_dof(w.dirichlet),
        model=w.model, p=w.p, C1=w.C1, D1=w.D1, f=per_dof(w.f), v=per_dof(w.v),
        eps=w.eps, extra=dict(w.extra))


def random_small(seed: int, dim: int, model: int, nx: int, ny: int, nz: int = 1,
                 jitter: float = 0.2, p: float = 3.0) -> Workload:
    """Small jittered structured mesh with random element orientation and vertex order,
    random Dirichlet dofs, random load and a random trial vector (for parity tests)."""
    if dim == 2:
        coords, elems = rect_tri(nx, ny)
        h = 1.0 / max(nx, ny)
    else:
        coords, elems = box_tet(nx, ny, nz)
        h = 1.0 / max(nx, ny, nz)
    nn, ne = coords.shape[0], elems.shape[0]
    interior = np.all((coords > 1e-12) & (coords < 1 - 1e-12), axis=1)
    jit = uniform(seed, np.arange(nn * dim), -jitter * h / 2, jitter * h / 2).reshape(nn, dim)
    coords = coords + jit * interior[:, None]
    # random vertex order inside each element (orientation flips)
    keys = splitmix64(seed + 101, np.arange(ne * (dim + 1))).reshape(ne, dim + 1)
    order = np.argsort(keys, axis=1)
    elems = np.take_along_axis(elems, order, axis=1).astype(np.int32)
    d = 1 if model == MODEL_PLAPLACE else dim
    dirichlet = (uniform(seed + 7, np.arange(nn * d), 0.0, 1.0) < 0.15).astype(np.uint8)
    f = uniform(seed + 11, np.arange(nn * d), -1.0, 1.0)
    if model == MODEL_PLAPLACE:
        v = uniform(seed + 13, np.arange(nn), -1.0, 1.0)
        C1 = D1 = 0.0
    else:
        v = coords.ravel() + uniform(seed + 13, np.arange(nn * d), -0.05 * h, 0.05 * h)
        C1, D1 = lame_c1_d1(1e4, 0.3)
    return Workload(
        name=f"random{dim}d_m{model}_s{seed}", dim=dim, d=d, coords=coords, elems=elems,
        dirichlet=dirichlet, model=model, p=p, C1=C1, D1=D1, f=f, v=v, eps=1e-6)


def config_workload(name: str) -> Workload:
    """The named synthetic workloads: 'C1' 2D p-Laplacian 64x64x2, 'C2' 2D Neo-Hookean
    1024x512x2, 'C3' 3D Neo-Hookean 128^3x6; suffix ':n' scales the grid (e.g. 'C3:32')."""
    base, _, arg = name.partition(":")
    if base == "C1":
        return plaplace_square(int(arg) if arg else 64)
    if base == "C2":
        if arg:
            k = int(arg)
            return neohooke_rect2d(2 * k, k)
        return neohooke_rect2d()
    if base == "C3":
        return neohooke_cube3d(int(arg) if arg else 128)
    raise ValueError(f"unknown workload {name!r}")
