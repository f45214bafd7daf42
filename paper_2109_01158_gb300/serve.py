"""Serving: continuous batching of energy + gradient requests over resident meshes.

A request asks for J(v) and grad J(v) on one mesh.  Meshes are precomputed once and stay
resident on the device (a catalogue keyed by model and size).  The server runs in real time
in the library (fe_server): requests arrive (Poisson process), wait in a FIFO, and are
admitted while their device bytes (the scratch of the batched kernels plus v and g) fit in
the HBM budget.  Each batch is evaluated in one persistent launch whatever its size, which
reads the vectors and writes the results straight in page-locked host memory and completes
each request on its own flag; requests that arrive while a batch runs join the next one,
which is prepared and enqueued while the GPU is still busy.  The one-at-a-time baseline runs
the same kernel with batches of one request, in arrival order.

Latency of a request = completion time - arrival time; the report gives p50/p99 latency,
requests/s and elements/s for both modes at the same offered load.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fem
from . import meshgen as mg

# ----------------------------------------------------------------------------------------
# Request stream (synthetic)
# ----------------------------------------------------------------------------------------

# Structured sizes of the catalogue: 2D n x n x 2 triangles, 3D n^3 x 6 tetrahedra.
SIZES_2D = [23, 32, 45, 64, 90, 128, 181, 256, 362, 512, 724, 1000]
SIZES_3D = [6, 8, 11, 15, 20, 28, 38, 52, 70]


@dataclass
class Request:
    rid: int
    key: tuple            # catalogue key: ("plap", p, n) / ("nh2", n) / ("nh3", n)
    arrival: float        # seconds after the start of the stream
    v: np.ndarray         # trial vector (host)
    ne: int = 0
    J: float = float("nan")
    g: np.ndarray | None = None
    t_start: float = float("nan")
    t_done: float = float("nan")

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def nearest(sizes, target, per_cell):
    return min(sizes, key=lambda n: abs(math.log(per_cell * n ** (2 if per_cell == 2 else 3)) - math.log(target)))


def request_keys(n_requests: int = 512, seed: int = 3, lo: float = 1e3, hi: float = 2e6):
    """Mix of the serving workload: 50% 2D p-Laplacian (p in {1.5, 2, 3}), 30% 2D Neo-Hookean,
    20% 3D Neo-Hookean; element counts log-uniform in [lo, hi] mapped to the nearest size of
    the catalogue.  All draws are SplitMix64 counters of `seed`."""
    u_kind = mg.uniform(seed, np.arange(n_requests), 0.0, 1.0)
    u_size = mg.uniform(seed, n_requests + np.arange(n_requests), 0.0, 1.0)
    u_p = mg.uniform(seed, 2 * n_requests + np.arange(n_requests), 0.0, 3.0)
    keys = []
    for k in range(n_requests):
        target = math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u_size[k])
        if u_kind[k] < 0.5:
            keys.append(("plap", (1.5, 2.0, 3.0)[min(int(u_p[k]), 2)], nearest(SIZES_2D, target, 2)))
        elif u_kind[k] < 0.8:
            keys.append(("nh2", nearest(SIZES_2D, target, 2)))
        else:
            keys.append(("nh3", nearest(SIZES_3D, target, 6)))
    return keys


def workload_for(key) -> mg.Workload:
    if key[0] == "plap":
        return mg.plaplace_square(key[2], p=key[1])
    if key[0] == "nh2":
        return mg.neohooke_rect2d(2 * key[1], key[1])
    return mg.neohooke_cube3d(key[1])


def request_vector(w: mg.Workload, rid: int, seed: int = 3) -> np.ndarray:
    """Per-request trial vector: the workload's v plus a small request-specific perturbation
    of the free dofs (SplitMix64 counters keyed by the request id)."""
    h = 1.0 / math.sqrt(max(w.ne, 1))
    pert = mg.uniform(seed * 1000003 + rid, np.arange(w.ndof), -1e-3 * h, 1e-3 * h)
    v = w.v + pert * (w.dirichlet == 0)
    return np.ascontiguousarray(v)


def poisson_arrivals(n: int, rate: float, seed: int = 3) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate (exponential gaps)."""
    u = mg.uniform(seed + 17, np.arange(n), 0.0, 1.0)
    return np.cumsum(-np.log1p(-u) / rate)


# ----------------------------------------------------------------------------------------
# Resident meshes
# ----------------------------------------------------------------------------------------

class Catalogue:
    """Precomputed meshes (FE_DF64) kept resident on the device, built on first use."""

    def __init__(self, device: int = 0):
        self.device = device
        self.meshes: dict = {}
        self.workloads: dict = {}

    def get(self, key):
        if key not in self.meshes:
            w = workload_for(key)
            self.workloads[key] = w
            self.meshes[key] = fem.FEMesh.from_workload(w, device=self.device, precisions=(fem.FE_DF64,))
        return self.meshes[key]

    def bytes(self) -> int:
        return sum(m.footprint() for m in self.meshes.values())


# ----------------------------------------------------------------------------------------
# Server
# ----------------------------------------------------------------------------------------

@dataclass
class ServeStats:
    mode: str
    n: int
    rate: float
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    max_batch: int
    steps: int
    req_per_s: float
    gelem_per_s: float
    launches: int
    latencies_ms: list = field(default_factory=list)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms")
        return d


class Server:
    """Real-time server over a catalogue of resident meshes.  The stream of requests is
    handed to the library's native server (fe_server) with each request's arrival time; its
    worker thread admits the arrived requests FIFO within the HBM budget and batches them
    (mode 'batched', up to max_batch per launch) or serves them one at a time ('serial'),
    with the same kernels either way."""

    def __init__(self, catalogue: Catalogue, hbm_budget: int = 8 << 30, max_batch: int = 256):
        self.cat = catalogue
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self._servers = {}      # mode -> fe_server, created on first use and kept
        self._pinned = {}       # id(request vector) -> page-locked (v, g) buffers

    def _buffers(self, r, mesh):
        """Page-locked copies of the request's vector and a page-locked result buffer (the
        server copies those by DMA directly), made once per request vector."""
        key = id(r.v)
        if key not in self._pinned:
            vt = torch.empty(mesh.ndof, dtype=torch.float64).pin_memory()
            gt = torch.zeros(mesh.ndof, dtype=torch.float64).pin_memory()
            vt.numpy()[:] = r.v
            self._pinned[key] = (r.v, vt, gt)
        _, vt, gt = self._pinned[key]
        return vt.numpy(), gt.numpy()

    def _server(self, mode):
        if mode not in self._servers:
            cap = self.max_batch if mode == "batched" else 1
            self._servers[mode] = fem.NativeServer(self.cat.device, self.budget, cap)
        return self._servers[mode]

    def close(self):
        for srv in self._servers.values():
            srv.close()
        self._servers.clear()
        self._pinned.clear()

    def run(self, requests: list, mode: str = "batched", keep_results: bool = True,
            lead_s: float = 0.05) -> ServeStats:
        """Serve `requests` (sorted by arrival, seconds from the start of the stream) in real
        time.  The stream starts lead_s after the server is created, so that every request is
        submitted before it arrives; latency = completion - arrival on the server clock."""
        assert mode in ("batched", "serial")
        for r in requests:           # meshes are resident before the stream starts
            self.cat.get(r.key)
        torch.cuda.synchronize(torch.device("cuda", self.cat.device))
        srv = self._server(mode)
        srv.reset_stats()
        # the callers' request and result buffers exist (page-locked) before the stream starts
        bufs = []
        for r in requests:
            mesh = self.cat.get(r.key)
            v, g = self._buffers(r, mesh)
            bufs.append((mesh, v, np.zeros(1), g))
        t0 = srv.now() + lead_s + 2e-5 * len(requests)
        sub = []
        for r, (mesh, v, J, g) in zip(requests, bufs):
            sub.append((r, srv.submit(mesh, v, J, g, t0 + r.arrival), J, g))
        for r, ticket, J, g in sub:
            st, ta, ts, td = srv.wait(ticket)
            r.t_start, r.t_done = ts - t0, td - t0
            if keep_results:
                r.J = float(J[0])
                r.g = g.copy()
        stats = srv.stats()
        wall = max(r.t_done for r in requests) if requests else 0.0
        lat = np.array([r.latency for r in requests]) * 1e3
        elems = sum(self.cat.get(r.key).ne for r in requests)
        rate = len(requests) / max(requests[-1].arrival, 1e-9)
        return ServeStats(mode, len(requests), rate, wall, float(np.percentile(lat, 50)),
                          float(np.percentile(lat, 99)), float(lat.mean()), stats["max_batch"],
                          stats["batches"], len(requests) / wall, elems / wall / 1e9,
                          stats["launches"], lat.tolist())


def make_requests(n: int = 512, seed: int = 3, rate: float = 1000.0, catalogue: Catalogue | None = None):
    keys = request_keys(n, seed)
    arrivals = poisson_arrivals(n, rate, seed)
    reqs = []
    cache = {}
    for k, (key, t) in enumerate(zip(keys, arrivals)):
        if key not in cache:
            cache[key] = workload_for(key) if catalogue is None else (catalogue.get(key), catalogue.workloads[key])[1]
        w = cache[key]
        reqs.append(Request(k, key, float(t), request_vector(w, k, seed), ne=w.ne))
    return reqs


def retime(requests, rate: float, seed: int = 3):
    """The same requests with arrival times of a Poisson process of rate `rate`."""
    arr = poisson_arrivals(len(requests), rate, seed)
    out = []
    for r, t in zip(requests, arr):
        out.append(Request(r.rid, r.key, float(t), r.v, ne=r.ne))
    return out


def serial_capacity(server: Server, requests) -> float:
    """Requests per second of back-to-back one-at-a-time service (all arrivals at t = 0)."""
    burst = [Request(r.rid, r.key, 0.0, r.v, ne=r.ne) for r in requests]
    st = server.run(burst, mode="serial", keep_results=False)
    return st.req_per_s


# ----------------------------------------------------------------------------------------
# Whole minimisations
# ----------------------------------------------------------------------------------------

@dataclass
class MinimizeRequest:
    """An L-BFGS minimisation of J on a resident mesh (FE_DF64; for Neo-Hookean usually with
    displacement input), from the device vector v0, to ||g||_inf <= gtol (times ||g0||_inf if
    relative).  arrival: seconds from the start of the stream."""
    rid: int
    mesh: object
    v0: torch.Tensor
    arrival: float
    gtol: float = 1e-6
    relative: bool = True
    t_admit: float = math.nan
    t_done: float = math.nan
    result: object = None

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclass
class MinimizeStats:
    mode: str
    n: int
    wall_s: float
    p50_s: float
    p99_s: float
    mean_s: float
    rounds: int
    max_active: int
    evaluations: int
    minimisations_per_s: float
    evaluations_per_s: float
    latencies_s: list = field(default_factory=list)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_s")
        return d


class MinimizeServer:
    """Continuous batching of whole minimisations.  Each admitted request is an L-BFGS job
    (minimize.LbfgsJob) whose iterate, gradient and curvature pairs stay on the device, with
    its directions computed by the library's L-BFGS kernels (fe_lbfgs).  A request is admitted
    once it has arrived and its device bytes (the batched kernels' scratch, the 2 (m + 1)
    vectors of the L-BFGS memory and 6 more of its mesh's size) fit in the HBM budget.  Every round evaluates the
    pending trial point of every admitted job in one batched launch (fe_batch, one persistent
    kernel whatever the number of jobs), feeds each job its J and g, and retires the jobs that have
    finished, which frees their bytes for the next arrivals.  Mode 'serial' admits one job at
    a time, in arrival order, with the same kernels.  A job's evaluations do not depend on the
    other jobs in the launch, so its iterates are the same in either mode."""

    def __init__(self, device: int = 0, hbm_budget: int = 4 << 30, max_active: int = 64, m: int = 10):
        from . import minimize
        self._mz = minimize
        self.device = torch.device("cuda", device)
        self.batch = fem.Batch(device)
        self.budget = int(hbm_budget)
        self.max_active = max_active
        self.m = m

    def job_bytes(self, mesh) -> int:
        return fem.Batch.work_bytes(mesh) + 256 + fem.LbfgsMemory.device_bytes(mesh.ndof, self.m) + 8 * mesh.ndof * 6

    def close(self):
        self.batch.close()

    def run(self, requests: list, mode: str = "batched") -> MinimizeStats:
        assert mode in ("batched", "serial")
        cap = self.max_active if mode == "batched" else 1
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        active = []            # (request, job, work tensor, bytes)
        used = 0
        rounds = evals = max_active = 0
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            while pending and len(active) < cap and pending[0].arrival <= now:
                r = pending[0]
                nb = self.job_bytes(r.mesh)
                if active and used + nb > self.budget:
                    break
                pending.pop(0)
                wb = fem.Batch.work_bytes(r.mesh)
                buf = torch.empty(wb + 256, dtype=torch.uint8, device=self.device)
                off = (-buf.data_ptr()) % 256
                job = self._mz.LbfgsJob(r.v0, m=self.m, gtol=r.gtol, relative=r.relative,
                                        eps_f=self._mz.EPS_F[fem.FE_DF64], device_memory=True)
                r.t_admit = now
                active.append((r, job, buf[off: off + wb], nb))
                used += nb
            if not active:
                wait = pending[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
                continue
            max_active = max(max_active, len(active))
            Js = torch.empty(len(active), dtype=torch.float64, device=self.device)
            items, gs = [], []
            for k, (r, job, work, _) in enumerate(active):
                g = torch.empty(r.mesh.ndof, dtype=torch.float64, device=self.device)
                items.append((r.mesh, job.trial().contiguous(), Js[k], g, work))
                gs.append(g)
            self.batch.run(items)
            self.batch.sync_status()
            # every job's J and g.d along its search direction in one read
            dirs = [job.search_direction() for _, job, _, _ in active]
            gds = [torch.dot(g, d) for g, d in zip(gs, dirs) if d is not None]
            host = torch.cat([Js] + ([torch.stack(gds)] if gds else [])).tolist()
            Jh, gdh = host[:len(active)], iter(host[len(active):])
            rounds += 1
            evals += len(active)
            still = []
            for (r, job, work, nb), J, g, d in zip(active, Jh, gs, dirs):
                job.feed(J, g, None if d is None else next(gdh))
                if job.done:
                    r.t_done = time.perf_counter() - t0
                    r.result = job.result()
                    used -= nb
                else:
                    still.append((r, job, work, nb))
            active = still
        wall = max(r.t_done for r in requests) if requests else 0.0
        lat = np.array([r.latency for r in requests])
        return MinimizeStats(mode, len(requests), wall, float(np.percentile(lat, 50)), float(np.percentile(lat, 99)),
                             float(lat.mean()), rounds, max_active, evals, len(requests) / wall, evals / wall,
                             lat.tolist())


def gravity_cube(n: int, scale: float = 1.0, device: int = 0):
    """A minimisation request's mesh: the 3D Neo-Hookean cube n^3 x 6, face x = 0 clamped,
    gravity (0, 0, -1e-2 scale), resident as FE_DF64 with displacement input; and u0 = 0."""
    w = mg.neohooke_cube3d(n)
    w.f = np.tile([0.0, 0.0, -1e-2 * scale], w.nn)
    w.v = w.coords.ravel().copy()
    mesh = fem.FEMesh.from_workload(w, device=device, precisions=(fem.FE_DF64,))
    mesh.set_input(fem.FE_INPUT_DISPLACEMENT)
    return mesh, torch.zeros(w.ndof, dtype=torch.float64, device=torch.device("cuda", device))


def make_minimize_requests(n: int = 16, sizes=(12, 16, 20, 24), rate: float = 20.0, seed: int = 5, device: int = 0,
                           gtol: float = 1e-6):
    """n minimisation requests: gravity cubes of sizes drawn from `sizes`, loads scaled by
    1 + k/n, Poisson arrivals of rate `rate` per second (seeded)."""
    pick = (mg.uniform(seed, np.arange(n), 0.0, len(sizes)).astype(np.int64)).clip(0, len(sizes) - 1)
    arr = poisson_arrivals(n, rate, seed)
    reqs = []
    for k in range(n):
        mesh, u0 = gravity_cube(int(sizes[pick[k]]), 1.0 + k / n, device)
        reqs.append(MinimizeRequest(k, mesh, u0, float(arr[k]), gtol=gtol, relative=True))
    return reqs
