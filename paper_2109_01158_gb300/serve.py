"""Serving: continuous batching of energy + gradient requests over resident meshes.

A request asks for J(v) and grad J(v) on one mesh.  Meshes are precomputed once and stay
resident on the device (a catalogue keyed by model and size).  The server runs in real time
in the library (fe_server): requests arrive (Poisson process), wait in a FIFO, and are
admitted while their device bytes (the scratch of the batched kernels plus v and g) fit in
the HBM budget.  Each batch is evaluated in three launches whatever its size; requests that
arrive while a batch runs join the next one, which is prepared and enqueued while the GPU
is still busy.  The one-at-a-time baseline runs the same kernels with batches of one
request, in arrival order.

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
