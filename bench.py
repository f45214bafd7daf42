#!/usr/bin/env python
"""Benchmark: energy + exact gradient throughput (G elements/s) on one GB300 per rank.

Workload (default): 3D compressible Neo-Hookean on the unit cube, 128^3 hexahedra x 6
tetrahedra (12,582,912 P1 tets, 2,146,689 nodes), face x=0 clamped, smooth displacement
0.05 sin(pi x) per component + U[-1e-4, 1e-4] noise (seed 2).  One step = one call of
fe_energy_gradient (node preparation, fused element kernel, patch gather).  The element
data of one step (1.5 GB) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f64|f32]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Prints one JSON line on rank 0.  For N > 1 (torchrun) every rank evaluates its own replica
of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes of one launch of the element kernel, per element and per node (each
# input read once in the paper's mesh layout: dim+1 shape gradients of dim entries, the
# volume, dim+1 node ids, and the nodal values gathered once).
ELEM_BYTES = {  # (dim, precision) -> (bytes per element, bytes per node)
    (3, "f64"): (12 * 8 + 8 + 4 * 4, 24),
    (2, "f64"): (6 * 8 + 8 + 3 * 4, 16),
    (3, "df64"): (12 * 8 + 8 + 4 * 4, 24),
    (2, "df64"): (6 * 8 + 8 + 3 * 4, 16),
    (3, "f32"): (12 * 4 + 4 + 4 * 4, 12),
    (2, "f32"): (6 * 4 + 4 + 3 * 4, 8),
}
# Whole-step algorithmic bytes add the patch CSR entries (4 B per element-node pair), the
# row pointers (4 B per node) and the gradient written in FP64.
STEP_EXTRA = {3: (4 * 4, 4 + 24), 2: (3 * 4, 4 + 16)}
# FP64 operations of the 3D Neo-Hookean energy + exact gradient per element, measured with
# ncu on the 64^3 x 6 element kernel: 81.18 DFMA (2 flops each) + 33.56 DADD + 45.07 DMUL
# thread instructions per tet.
F64_FLOPS_PER_TET = 240.98


def fp64_probe(dev_index: int):
    """The FP64 issue rates of this GPU (fe_fp64_rate: operations per SM clock per SM) and its
    SM count; run before the timed regions."""
    import torch
    from paper_2109_01158_gb300 import fem
    rate, ghz = fem.fp64_rate(dev_index, fem.FE_RATE_DFMA)
    add_rate, _ = fem.fp64_rate(dev_index, fem.FE_RATE_DADD)
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    return {"dfma_per_clk_per_sm": rate, "dadd_per_clk_per_sm": add_rate, "sms": sms, "probe_sm_ghz": ghz}


def fp64_peak_tflops(probe: dict, sm_max_mhz):
    """FP64 peak from the measured DFMA rate, the SM count and the maximum SM clock
    (nvidia-smi; the probe's own clock when that is unknown): 2 flops x rate x SMs x clock."""
    mhz = sm_max_mhz if sm_max_mhz else probe["probe_sm_ghz"] * 1e3
    peak = 2.0 * probe["dfma_per_clk_per_sm"] * probe["sms"] * mhz * 1e6 / 1e12
    return peak, dict(probe, sm_mhz=mhz, formula="2 flops x measured DFMA/clk/SM x SMs x max SM clock")


# What one step runs in each precision (for the variants' records).
VARIANT_KERNELS = {
    "f64": "k_node_prep + k_elem_f64 (local forces to HBM) + k_gather_bulk (patch sums)",
    "df64": "k_node_prep_df + k_elem_df (local forces to HBM) + k_gather_bulk (patch sums)",
    "f32": "k_pairs32 (node pairs) + k_tile_f32 (elements and patch sums in shared memory, one persistent "
           "warp-specialised block per SM) + k_tile_shared (nodes on tile boundaries)",
}

# DRAM traffic of the element kernels per launch, from an ncu capture (profiles/): valid only
# while the kernel's sources hash to the value recorded with the capture.
ORDER_NAMES = {0: "as generated", 1: "Morton", 2: "reverse Cuthill-McKee"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
L2_BYTES = 129 << 20        # GB300 L2 (for the flush decision)
FLUSH_BYTES = 256 << 20     # a write of this size evicts L2

KERNEL_SOURCES = {
    "f64": ["fe_eval_f64.cu", "fe_internal.cuh", "phi_f64.cuh", "phi_table_f64.h"],
    "df64": ["fe_eval_df64.cu", "elem_df.cuh", "df64.cuh", "fe_internal.cuh"],
    "f32": ["fe_eval_f32.cu", "elem_f32.cuh", "tile_common.cuh", "fe_tiles.cu", "df64.cuh", "fe_internal.cuh",
            "async_copy.cuh"],
}


def sources_sha256(prec):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[prec]:
        with open(os.path.join(ROOT, "paper_2109_01158_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_record(prec, dim):
    """The ncu capture of the element kernel, or None when there is none for this kernel or
    its sources changed since."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)[prec]
    except Exception:
        return None
    if rec.get("dim") != dim or rec.get("sources_sha256") != sources_sha256(prec):
        return None
    return rec


def recorded_traffic(prec, dim, ne):
    """DRAM bytes per launch of the element kernel scaled to ne elements (or None)."""
    rec = traffic_record(prec, dim)
    return None if rec is None else float(rec["bytes_per_element"]) * ne


def load_peaks():
    try:
        with open(MEASURED_PEAKS) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------------------

def dist_setup(ngpus):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------------------

def oracle_sample(w, fraction):
    """A bounded sample of the workload: its first `fraction` of elements (whole layers of
    the structured mesh) on the full node set."""
    import numpy as np
    from paper_2109_01158_gb300 import meshgen as mg
    m = max(1, int(w.ne * fraction))
    return mg.Workload(w.name + f"_first{m}", w.dim, w.d, w.coords, np.ascontiguousarray(w.elems[:m]),
                       w.dirichlet, w.model, p=w.p, C1=w.C1, D1=w.D1, f=w.f, v=w.v, eps=w.eps)


def time_oracle(ws, reps):
    import oracle
    om = oracle.OracleMesh(ws)
    om.energy(ws.v)            # page in the working set once
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        om.energy(ws.v)
        om.gradient_exact(ws.v)
        ts.append(time.perf_counter() - t0)
    return ts


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_range_worker(task):
    """One process of the all-cores timing: the oracle's energy + exact gradient over elements
    [lo, hi) of the workload (its own single-threaded C code), started together with the other
    processes at a barrier; returns (start, end) wall-clock times of its `reps` evaluations."""
    name, lo, hi, reps, start_barrier = task
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2109_01158_gb300 import meshgen as mg
    w = mg.config_workload(name)
    ws = mg.Workload(w.name + f"_{lo}_{hi}", w.dim, w.d, w.coords, np.ascontiguousarray(w.elems[lo:hi]),
                     w.dirichlet, w.model, p=w.p, C1=w.C1, D1=w.D1, f=w.f, v=w.v, eps=w.eps)
    om = oracle.OracleMesh(ws)
    om.energy(ws.v)                       # page in the working set once
    start_barrier.wait()
    t0 = time.time()
    for _ in range(reps):
        om.energy(ws.v)
        om.gradient_exact(ws.v)
    return t0, time.time()


def time_oracle_all_cores(name, ne, reps=2, procs=None):
    """The oracle on every host core: the mesh's elements split into one contiguous range per
    process (spawned, one thread each), all started at once; whole-job elements/s over the
    wall time from the first start to the last end."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        bar = mgr.Barrier(procs)
        cuts = [ne * k // procs for k in range(procs + 1)]
        tasks = [(name, cuts[k], cuts[k + 1], reps, bar) for k in range(procs)]
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_range_worker, tasks)
    wall = max(t1 for _, t1 in res) - min(t0 for t0, _ in res)
    return ne * reps / wall / 1e9, procs, wall


def run_reference(args, rank, world):
    from paper_2109_01158_gb300 import meshgen as mg
    if rank != 0:
        return None
    w = mg.config_workload(args.workload)
    ws = oracle_sample(w, args.sample_fraction)
    ts = time_oracle(ws, args.warmup + args.steps)[args.warmup:]
    total = sum(ts)
    value = ws.ne * len(ts) / total / 1e9
    sample = (f"first {ws.ne} of {w.ne} elements of {w.name} ({args.sample_fraction:g} of the mesh, "
              f"whole element layers), energy + exact gradient per step, single thread")
    line = {
        "impl": "reference", "metric": "energy+grad throughput", "value": value, "unit": "Gelem/s",
        "n_gpus": 0, "steps": len(ts), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, "f64"),
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------

def workload_config(w, precision):
    return {
        "workload": (f"{w.name}: {'3D' if w.dim == 3 else '2D'} "
                     f"{'compressible Neo-Hookean' if w.model == 1 else f'p-Laplacian p={w.p:g}'}, "
                     f"{w.ne} P1 elements, {w.nn} nodes, {w.ndof} dofs; energy + exact gradient"),
        "elements": w.ne, "nodes": w.nn, "dofs": w.ndof, "precision": precision,
        "l2": "inputs larger than L2 (element data of one step > 129 MB), no flush",
        "parallelism": "replicas",
    }


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2109_01158_gb300 import fem
    from paper_2109_01158_gb300 import meshgen as mg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = mg.config_workload(args.workload)
    if args.shuffle_nodes:
        w = mg.shuffle_nodes(w, 4)
    code = {"f64": fem.FE_F64, "f32": fem.FE_F32_COMP, "df64": fem.FE_DF64}
    others = [k for k in ("df64", "f64", "f32") if k != args.precision]
    precs = tuple(code[k] for k in [args.precision] + others)
    gm = fem.FEMesh.from_workload(w, device=local, order=args.order, precisions=precs)
    v = torch.from_numpy(w.v).to(dev)
    J = torch.empty((), dtype=torch.float64, device=dev)
    g = torch.empty(w.ndof, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def steps(n):
        for _ in range(n):
            gm.energy_gradient(v, J, g)

    # Inputs smaller than twice L2 (or --flush-l2): every timed step is preceded by a 256 MB
    # write that evicts L2, and only the steps are timed (an event pair around each).
    step_data = w.ne * ELEM_BYTES[(w.dim, args.precision)][0] + w.nn * ELEM_BYTES[(w.dim, args.precision)][1]
    flush = args.flush_l2 or step_data < 2 * L2_BYTES
    flush_buf = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev) if flush else None

    def timed(n, profile=False):
        if profile:
            gm.profile(True)
        barrier(world)
        torch.cuda.synchronize(dev)
        l0 = gm.launch_count()
        if flush_buf is None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            steps(n)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
        else:
            evs = []
            for _ in range(n):
                flush_buf.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gm.energy_gradient(v, J, g)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
            ms = sum(a.elapsed_time(b) for a, b in evs)
        barrier(world)
        prof = gm.profile_read() if profile else None
        if profile:
            gm.profile(False)
        return ms, gm.launch_count() - l0, prof

    probe = fp64_probe(local) if (args.precision == "f64" and w.dim == 3 and w.model == mg.MODEL_NEOHOOKE) else None
    steps(args.warmup)
    assert gm.sync_status() == fem.FE_OK, "domain error in the benchmark workload"
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    ms, launches, prof = timed(args.steps, profile=True)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, world, dev)
    ms_step = ms / args.steps
    value = w.ne * args.steps * world / (ms / 1e3) / 1e9

    # roofline of the dominant kernel (the element kernel), timed by events on its stream
    hbm_peak, peak_kind = load_peaks()
    prec = args.precision
    elem_ms = prof["element"][0] / max(prof["element"][1], 1)
    bpe, bpn = ELEM_BYTES[(w.dim, prec)]
    elem_bytes = w.ne * bpe + w.nn * bpn
    xe, xn = STEP_EXTRA[w.dim]
    step_bytes = elem_bytes + w.ne * xe + w.nn * xn
    hbm_achieved = elem_bytes / (elem_ms / 1e3) / 1e9
    if prec == "f64" and w.dim == 3 and w.model == mg.MODEL_NEOHOOKE:
        achieved = F64_FLOPS_PER_TET * w.ne / (elem_ms / 1e3) / 1e12
        f64_peak, f64_probe = fp64_peak_tflops(probe, clocks.get("sm_max_mhz"))
        roof = {"bound": "alu", "achieved": achieved, "peak": f64_peak, "unit": "TFLOP/s",
                "frac": achieved / f64_peak, "traffic": None,
                "peak_kind": "derived FP64 from a measured DFMA rate", "fp64_probe": f64_probe,
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": hbm_achieved / hbm_peak, "peak_kind": peak_kind}}
    else:
        roof = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind}
    roof["traffic"] = recorded_traffic(prec, w.dim, w.ne)
    trec = traffic_record(prec, w.dim)
    if trec is not None:
        sc = w.ne / trec["elements"]
        roof["traffic_read"] = trec["dram_bytes_read"] * sc
        roof["traffic_write"] = trec["dram_bytes_write"] * sc
        roof["traffic_note"] = (
            "scaled by the element count from an ncu capture of %s on %s; reads are the algorithmic element "
            "and node bytes (no re-reads); writes are the local forces (dim+1)*d per element (FP64 and "
            "double-float; the FP32 tiles keep them on chip), undercounted by the lines still in L2 when the "
            "captured launch ended" % (trec["kernel"], trec["workload"]))
    roof["kernel"] = {"f64": "k_elem_f64", "df64": "k_elem_df", "f32": "k_tile_f32"}[prec] + " (energy+gradient)"
    roof["kernel_ms"] = elem_ms
    roof["algorithmic_bytes_per_launch"] = elem_bytes
    stages = {k: {"ms_per_launch": t / n if n else 0.0, "launches": n} for k, (t, n) in prof.items() if n}

    # end to end through the public API with host buffers (pinned), copies inside the region.
    # fe_energy_gradient_host_async overlaps the copies of step k + 1 in and of step k - 1 out
    # with step k; the timed region ends when the last step's J and g are in host memory.
    vh = torch.from_numpy(w.v).pin_memory()
    gh = [torch.empty(w.ndof, dtype=torch.float64).pin_memory() for _ in range(2)]
    Jh = torch.empty((2, 1), dtype=torch.float64).pin_memory()
    vh_np, gh_np, Jh_np = vh.numpy(), [t.numpy() for t in gh], Jh.numpy()
    e2e_steps = max(10, args.steps)

    def host_steps(n, pipelined):
        for k in range(n):
            if pipelined:
                gm.energy_gradient_host_async(vh_np, Jh_np[k % 2], gh_np[k % 2])
            else:
                gm.energy_gradient_host(vh_np, gh_np[0])
        if pipelined:
            gm.host_wait()

    e2e = {}
    for pipelined in (False, True):
        host_steps(3, pipelined)
        barrier(world)
        t0 = time.perf_counter()
        host_steps(e2e_steps, pipelined)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e["value" if pipelined else "serial_value"] = w.ne * e2e_steps * world / e2e_s / 1e9
    e2e.update({"unit": "Gelem/s", "h2d_bytes_per_step": w.ndof * 8, "d2h_bytes_per_step": w.ndof * 8 + 8,
                "api": "fe_energy_gradient_host_async (pipelined, two device slots)",
                "serial_api": "fe_energy_gradient_host (one call at a time)"})
    e2e = {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "api",
                               "serial_value", "serial_api")}
    if flush:
        e2e["l2"] = ("steps back to back, L2 not evicted between them (unlike value): the inputs fit in L2, "
                     "so this can exceed value")

    # the other precisions (same mesh), for context
    variants = {}
    for other in others:
        gm.set_precision(code[other])
        steps(3)
        nst = max(5, args.steps // 4)
        oms, _, oprof = timed(nst, profile=True)
        o_elem = oprof["element"][0] / max(oprof["element"][1], 1)
        ob, on = ELEM_BYTES[(w.dim, other)]
        o_step_bytes = w.ne * (ob + xe) + w.nn * (on + xn)
        variants[other] = {"value": w.ne * nst / (oms / 1e3) / 1e9, "unit": "Gelem/s",
                           "ms_per_step": oms / nst, "element_kernel_ms": o_elem,
                           "element_hbm_frac": (w.ne * ob + w.nn * on) / (o_elem / 1e3) / 1e9 / hbm_peak,
                           "step_algorithmic_bytes": o_step_bytes,
                           "step_hbm_frac": o_step_bytes / (oms / nst / 1e3) / 1e9 / hbm_peak,
                           "stages_ms": {k: t / n for k, (t, n) in oprof.items() if n},
                           "kernels": VARIANT_KERNELS.get(other, "")}
    gm.set_precision(code[prec])

    # Hessian-vector products (FP64) on the same mesh and state, for context
    x = torch.from_numpy(mg.uniform(80, np.arange(w.ndof), -1.0, 1.0)).to(dev)
    Hx = torch.empty(w.ndof, dtype=torch.float64, device=dev)
    for _ in range(3):
        gm.hessian_vector(v, x, out=Hx)
    nh = max(5, args.steps // 4)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nh):
        gm.hessian_vector(v, x, out=Hx)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    hms = e0.elapsed_time(e1) / nh
    variants["f64_hessian_vector"] = {"value": w.ne / (hms / 1e3) / 1e9, "unit": "Gelem/s", "ms_per_call": hms}

    # the energy alone (the forward of the autograd function; Table 2 times this), FP64
    if gm.precision != fem.FE_F64:
        gm.set_precision(fem.FE_F64)
    for _ in range(3):
        gm.energy(v)
    ne_steps = max(5, args.steps // 4)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(ne_steps):
        gm.energy(v)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ems = e0.elapsed_time(e1) / ne_steps
    variants["f64_energy"] = {"value": w.ne / (ems / 1e3) / 1e9, "unit": "Gelem/s", "ms_per_call": ems}
    gm.set_precision(code[prec])

    # one trust-region Newton step's inner solve: 50 Steihaug CG steps on the device (products
    # from the per-solve cache of the Hessian terms at v), FP64
    _, gv = gm.energy_gradient(v)
    gm.cg_steihaug(v, gv, 1e30, 0.0, 5)
    ncg = 50
    torch.cuda.synchronize(dev)
    e0.record(stream)
    _, _, kcg, _ = gm.cg_steihaug(v, gv, 1e30, 0.0, ncg)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    cms = e0.elapsed_time(e1)
    variants["f64_cg_steihaug"] = {"value": w.ne * kcg / (cms / 1e3) / 1e9, "unit": "Gelem/s",
                                   "ms_per_cg_step": cms / max(kcg, 1), "cg_steps": kcg,
                                   "note": "products per second x elements; includes the per-solve preparation"}

    # the paper's central-difference gradient over patches (Sec. 6.1), every dof, FP64:
    # 2 (dim + 1) d density evaluations per element
    if gm.precision != fem.FE_F64:
        gm.set_precision(fem.FE_F64)
    for _ in range(2):
        gm.gradient_fd(v, 1e-6)
    nf = max(3, args.steps // 20)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(nf):
        gm.gradient_fd(v, 1e-6)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fms = e0.elapsed_time(e1) / nf
    assert gm.sync_status() == fem.FE_OK
    n_w = 2 * (w.dim + 1) * w.d
    variants["f64_fd_gradient"] = {"value": w.ne / (fms / 1e3) / 1e9, "unit": "Gelem/s", "ms_per_call": fms,
                                   "density_evaluations_per_element": n_w, "eps": 1e-6}
    gm.set_precision(code[prec])

    line = {
        "metric": "energy+grad throughput", "value": value, "unit": "Gelem/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": dict(workload_config(w, prec), node_order=ORDER_NAMES[args.order],
                       **({"l2": "L2 evicted before every timed step (256 MB write, not timed)"} if flush else {})),
        "roofline": roof,
        "step_hbm": {"algorithmic_bytes": step_bytes,
                     "achieved_gbs": step_bytes / (ms_step / 1e3) / 1e9,
                     "frac": step_bytes / (ms_step / 1e3) / 1e9 / hbm_peak},
        "stages": stages, "variants": variants,
        "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0 and not args.no_serve:
        line["serving"] = run_serving(args, local)
    if rank == 0 and world == 1 and not args.no_minimize:
        # the bounded set by default (about 30 s); the paper's minimisation benchmarks with --minimize
        line["minimize"] = run_minimize(args, local, full=args.minimize)
    if rank == 0 and args.paper_tables:
        line["paper_tables"] = run_paper_tables(args, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ws = oracle_sample(w, args.sample_fraction)
        ts = time_oracle(ws, 2)
        best = min(ts)
        line["cpu_baseline"] = {
            "value": ws.ne / best / 1e9, "unit": "Gelem/s", "cores": 1, "kind": "oracle",
            "sample": (f"first {ws.ne} of {w.ne} elements (whole element layers), energy + exact "
                       f"gradient, best of 2, single thread"),
            "cpu_model": cpu_model()}
        try:
            allv, procs, wall = time_oracle_all_cores(args.workload, w.ne, reps=2)
            line["cpu_baseline"]["all_cores"] = {
                "value": allv, "unit": "Gelem/s", "cores": procs, "kind": "oracle",
                "sample": (f"all {w.ne} elements, split into {procs} contiguous element ranges, one "
                           f"spawned process per core running the oracle's single-threaded C code; "
                           f"energy + exact gradient twice each, {wall:.2f} s wall from the first start to "
                           f"the last end"),
                "cpu_model": line["cpu_baseline"]["cpu_model"]}
        except Exception as exc:   # a host without spawn support or memory for every process
            line["cpu_baseline"]["all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"}
    gm.close()
    return line if rank == 0 else None


def run_serving(args, device):
    """Continuous batching vs one request at a time on the same GPU and kernels (FE_DF64):
    512 requests (50% 2D p-Laplacian p in {1.5, 2, 3}, 30% 2D Neo-Hookean, 20% 3D
    Neo-Hookean, 1e3-2e6 elements log-uniform, seed 3), Poisson arrivals at 0.5, 0.8, 0.95,
    1.5 and 3 times the measured one-at-a-time capacity; p50/p99 latency = completion -
    arrival."""
    from paper_2109_01158_gb300 import serve
    t0 = time.perf_counter()
    cat = serve.Catalogue(device)
    reqs = serve.make_requests(args.serve_requests, seed=3, rate=1.0, catalogue=cat)
    setup_s = time.perf_counter() - t0
    server = serve.Server(cat, hbm_budget=args.serve_budget_gb << 30)
    warm = [serve.Request(r.rid, r.key, 0.0, r.v, ne=r.ne) for r in reqs[:64]]
    server.run(warm, mode="serial", keep_results=False)     # warm-up of both native servers
    server.run(warm, mode="batched", keep_results=False)
    cap = serve.serial_capacity(server, reqs)
    out = {"requests": len(reqs), "precision": "df64", "catalogue_meshes": len(cat.meshes),
           "resident_bytes": cat.bytes(), "setup_s": setup_s, "serial_capacity_req_s": cap,
           "hbm_budget_bytes": server.budget, "loads": []}
    burst = [serve.Request(r.rid, r.key, 0.0, r.v, ne=r.ne) for r in reqs]
    out["batched_capacity_req_s"] = server.run(burst, mode="batched", keep_results=False).req_per_s
    for load in (0.5, 0.8, 0.95, 1.5, 3.0):
        rate = load * cap
        rec = {"load": load, "rate_req_s": rate}
        for mode in ("batched", "serial"):
            st = server.run(serve.retime(reqs, rate, seed=3), mode=mode, keep_results=False)
            rec[mode] = {k: st.as_dict()[k] for k in ("p50_ms", "p99_ms", "mean_ms", "req_per_s",
                                                       "gelem_per_s", "max_batch", "steps", "wall_s")}
        out["loads"].append(rec)
    server.close()
    return out


# Tables 2 and 3 of the paper (twisted bar, levels 1-5): seconds for 10 evaluations on an
# M1 in MATLAB -- energy; exact gradient; central-difference gradient.
PAPER_TABLE2_10X = {1: 0.01, 2: 0.02, 3: 0.08, 4: 0.76, 5: 12.82}
PAPER_TABLE3_EXACT_10X = {1: 0.12, 2: 0.14, 3: 1.18, 4: 12.47, 5: 487.34}
PAPER_TABLE3_CD_10X = {1: 0.08, 2: 0.15, 3: 1.51, 4: 15.64, 5: 533.24}


def run_paper_tables(args, device):
    """The evaluations of Benchmarks 2 and 3 on their own meshes (the twisted bar, levels 1-5,
    FP64): energy, exact gradient and central-difference gradient (eps = 1e-6), each timed
    over 10 calls by events after warm-up, beside the paper's times for 10 evaluations."""
    import torch
    from paper_2109_01158_gb300 import fem
    from paper_2109_01158_gb300 import meshgen as mg
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for level in range(1, 6):
        w = mg.twisted_bar(level)
        gm = fem.FEMesh.from_workload(w, device=device)
        v = torch.from_numpy(w.v).to(dev)
        calls = {"energy": lambda: gm.energy(v), "gradient_exact": lambda: gm.gradient_exact(v),
                 "gradient_cd": lambda: gm.gradient_fd(v, 1e-6)}
        rec = {"level": level, "tets": w.ne, "free_dofs": int((w.dirichlet == 0).sum())}
        for name, fn in calls.items():
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            rec[name + "_10x_s"] = e0.elapsed_time(e1) / 1e3
        assert gm.sync_status() == fem.FE_OK
        rec["J_grad"] = float(gm.energy(v).item()) if w.f is None else None
        rec["paper_10x_s"] = {"energy": PAPER_TABLE2_10X[level], "gradient_exact": PAPER_TABLE3_EXACT_10X[level],
                              "gradient_cd": PAPER_TABLE3_CD_10X[level]}
        rows.append(rec)
        del gm
    return {"workload": "Benchmarks 2 and 3: twisted bar, 80*2^(L-1) x 2^L x 2^L hexes x 6 tets, FP64, "
                        "10 calls each", "levels": rows,
            "paper": "MATLAB R2021a on an M1 MacBook Air (Sec. 7.3); other hardware, context only"}


def served_minimisations(device):
    """Whole minimisations served by continuous batching: 16 gravity-cube requests
    (12^3..24^3 x 6, loads 1 + k/16), Poisson arrivals at 40/s; batched rounds vs one request at
    a time, and whether every result is bitwise the same in both."""
    import torch
    from paper_2109_01158_gb300 import serve
    msrv = serve.MinimizeServer(device)
    for mode in ("serial", "batched"):   # untimed warm-up of both modes (first-use costs)
        msrv.run(serve.make_minimize_requests(2, rate=40.0, device=device), mode)
    served = {}
    for mode in ("serial", "batched"):
        reqs = serve.make_minimize_requests(16, rate=40.0, device=device)
        served[mode] = (msrv.run(reqs, mode), reqs)
    msrv.close()
    same = all(a.result.J == b.result.J and torch.equal(a.result.v, b.result.v)
               for a, b in zip(served["batched"][1], served["serial"][1]))
    return {
        "workload": "16 L-BFGS requests, 3D Neo-Hookean gravity cubes 12^3..24^3 x 6, Poisson arrivals 40/s, "
                    "||g||_inf <= 1e-6 ||g0||_inf, double-float kernels",
        "batched": served["batched"][0].as_dict(), "serial": served["serial"][0].as_dict(),
        "results_identical_alone_and_in_the_mix": same,
        "converged": all(r.result.converged for r in served["batched"][1])}


def run_minimize(args, device, full=True):
    """End-to-end minimisation: 3D Neo-Hookean 64^3 x 6 tetrahedra (1,572,864), face x = 0
    clamped, gravity f = (0, 0, -1e-2), E = 1e4, nu = 0.3, from v = X; L-BFGS (m = 10) on the
    displacement u = v - X (FE_INPUT_DISPLACEMENT) until
    ||g||_inf <= 1e-6 ||g_0||_inf, driven by the exact-gradient kernels (double-float, FP64,
    FP32) and by the FP64 central-difference gradient (eps = 1e-6), and eight instances (load scaled by
    1 + k/8, 32^3 x 6 each) in lockstep through the batched kernels."""
    import numpy as np
    import torch
    from paper_2109_01158_gb300 import fem
    from paper_2109_01158_gb300 import meshgen as mg
    from paper_2109_01158_gb300.minimize import (batch_evaluator, lbfgs, lbfgs_batched, mesh_cg, mesh_evaluator,
                                                 mesh_hvp, nested_newton, newton_cg, torsion_continuation)
    n = args.minimize_n
    dev = torch.device("cuda", device)

    def problem(scale=1.0, size=n):
        w = mg.neohooke_cube3d(size)
        w.f = np.tile([0.0, 0.0, -1e-2 * scale], w.nn)
        w.v = w.coords.ravel().copy()
        return w

    w = problem()
    gm = fem.FEMesh.from_workload(w, device=device, precisions=(fem.FE_DF64, fem.FE_F64, fem.FE_F32_COMP))
    gm.set_input(fem.FE_INPUT_DISPLACEMENT)
    v0 = torch.zeros(w.ndof, dtype=torch.float64, device=dev)     # u = 0, i.e. v = X
    out = {"workload": f"neohooke3d_{n}^3x6 gravity (0,0,-1e-2), {w.ne} tets, {w.ndof} dofs",
           "criterion": "||g||_inf <= 1e-6 ||g_0||_inf", "unknown": "displacement u = v - X",
           "runs": {}}
    # L-BFGS pairs and directions in the library's kernels (fe_lbfgs); one run with the same
    # recursion in torch vector operations for comparison
    runs = [("df64_exact", fem.FE_DF64, "exact", True), ("f64_exact", fem.FE_F64, "exact", True)]
    if full:
        runs += [("f64_exact_torch_memory", fem.FE_F64, "exact", False), ("f32_exact", fem.FE_F32_COMP, "exact", True),
                 ("f64_fd", fem.FE_F64, "fd", True)]
    # untimed warm-up of every method (a few iterations): the first use of a kernel in a
    # process loads its module, which would otherwise be timed with the first run
    for name, prec, grad, devmem in runs:
        gm.set_precision(prec)
        lbfgs(mesh_evaluator(gm, grad, eps=1e-6), v0, gtol=1e-6, relative=True, max_iter=3, device_memory=devmem)
    gm.set_precision(fem.FE_F64)
    newton_cg(mesh_evaluator(gm), mesh_hvp(gm), v0, gtol=1e-6, relative=True, cg=mesh_cg(gm), max_iter=1)
    torch.cuda.synchronize(dev)
    for name, prec, grad, devmem in runs:
        gm.set_precision(prec)
        r = lbfgs(mesh_evaluator(gm, grad, eps=1e-6), v0, gtol=1e-6, relative=True, max_iter=args.minimize_iters,
                  device_memory=devmem)
        out["runs"][name] = {"J": r.J, "iters": r.iters, "evals": r.evals, "converged": r.converged,
                             "seconds": r.seconds, "gnorm": r.gnorm, "g0": r.history[0][1]}
    # trust-region Newton-CG on the FP64 Hessian-vector products (device-resident inner CG)
    gm.set_precision(fem.FE_F64)
    r = newton_cg(mesh_evaluator(gm), mesh_hvp(gm), v0, gtol=1e-6, relative=True, cg=mesh_cg(gm))
    out["runs"]["f64_newton_cg"] = {"J": r.J, "iters": r.iters, "evals": r.evals, "hessian_vector_products": r.hvps,
                                    "converged": r.converged, "seconds": r.seconds, "gnorm": r.gnorm,
                                    "g0": r.history[0][1]}
    ref = out["runs"]["df64_exact"]["J"]
    for rec in out["runs"].values():
        rec["J_rel_diff_vs_df64"] = abs(rec["J"] - ref) / abs(ref)
    # eight instances of the problem on 32^3 x 6 (load scaled by 1 + k/8) in lockstep: one
    # batched launch per line-search round evaluates every active instance's trial point
    nl = max(n // 2, 4)
    ws = [problem(1.0 + k / 8.0, nl) for k in range(8)]
    meshes = [fem.FEMesh.from_workload(wk, device=device, precisions=(fem.FE_DF64,)) for wk in ws]
    for m in meshes:
        m.set_input(fem.FE_INPUT_DISPLACEMENT)
    batch = fem.Batch(device)
    t_lock = time.perf_counter()
    rs = lbfgs_batched(batch_evaluator(batch, meshes, device),
                       [torch.zeros(wk.ndof, dtype=torch.float64, device=dev) for wk in ws],
                       gtol=1e-6, relative=True, max_iter=args.minimize_iters, device_memory=True)
    t_lock = time.perf_counter() - t_lock
    out["lockstep_8_instances"] = {
        "workload": f"8 x neohooke3d_{nl}^3x6 gravity, loads 1 + k/8, double-float kernels, one batched launch "
                    f"per line-search round",
        "iters": [r.iters for r in rs], "converged": all(r.converged for r in rs), "seconds": t_lock}
    if not full:
        out["served_minimisations"] = served_minimisations(device)
        return out
    # Benchmark 4: the torsion continuation (24 minimisations) on the level-3 bar, FP64
    # kernels with trust-region Newton-CG, against the minimal energies the paper prints
    paper3 = {3: 1.4631, 6: 5.8533, 9: 13.1735, 12: 23.4286, 15: 36.6236, 18: 52.7641, 21: 71.7883, 24: 93.7238}
    wb = mg.twisted_bar(3)
    gb = fem.FEMesh.from_workload(wb, device=device)
    tors = {"workload": f"Benchmark 4 torsion, bar level 3 ({wb.ne} tets, "
                        f"{int((wb.dirichlet == 0).sum())} free dofs), t = 1..24, alpha = 8 pi t / 24",
            "steps": []}
    t_start = time.perf_counter()
    for t, r in torsion_continuation(mesh_evaluator(gb), mesh_hvp(gb), torch.from_numpy(wb.coords).to(dev),
                                     torch.from_numpy(wb.dirichlet.astype(np.int64)).to(dev), cg=mesh_cg(gb),
                                     eta_max=0.5):
        rec = {"t": t, "J": r.J, "iters": r.iters, "hessian_vector_products": r.hvps, "converged": r.converged,
               "seconds": r.seconds}
        if t in paper3:
            rec["J_paper"] = paper3[t]
        tors["steps"].append(rec)
    tors["seconds"] = time.perf_counter() - t_start
    out["torsion_benchmark4_level3"] = tors
    # Benchmark 6: the L-shape p-Laplacian (p = 3, f = -10) at level 8 (784,385 free dofs),
    # componentwise density (the reading of the printed minima), FP64 Newton-CG: from v = 0
    # as the paper, and by nested iteration over levels 1..8
    lmeshes = []
    for L in range(1, 9):
        lc, le, lb = mg.lshape_tri(L)
        wl = mg.Workload(f"lshape{L}", 2, 1, lc, le, lb.astype(np.uint8), mg.MODEL_PLAPLACE_LP, p=3.0,
                         f=np.full(lc.shape[0], -10.0), v=np.zeros(lc.shape[0]))
        lmeshes.append((wl, fem.FEMesh.from_workload(wl, device=device)))
    wl, gl = lmeshes[-1]
    r = newton_cg(mesh_evaluator(gl), mesh_hvp(gl), torch.zeros(wl.nn, dtype=torch.float64, device=dev),
                  gtol=1e-10, max_iter=5000, cg=mesh_cg(gl))
    t_nest = time.perf_counter()
    rn = nested_newton([(mesh_evaluator(g), mesh_hvp(g), mesh_cg(g), w.coords, w.elems) for w, g in lmeshes],
                       torch.zeros(lmeshes[0][0].nn, dtype=torch.float64, device=dev), gtol=1e-10, max_iter=5000)
    t_nest = time.perf_counter() - t_nest
    out["lshape_benchmark6_level8"] = {
        "workload": f"Benchmark 6 L-shape level 8 ({wl.ne} triangles, {int((wl.dirichlet == 0).sum())} free dofs)",
        "J": r.J, "J_paper": -8.1649, "iters": r.iters, "hessian_vector_products": r.hvps,
        "converged": r.converged, "seconds": r.seconds,
        "nested": {"J": rn[-1].J, "iters_per_level": [x.iters for x in rn],
                   "hessian_vector_products_per_level": [x.hvps for x in rn],
                   "converged": all(x.converged for x in rn), "seconds_level8": rn[-1].seconds,
                   "seconds_total": t_nest},
        "paper": "617.92 s, 22 trust-region iterations (exact gradient; MATLAB on an M1)"}
    out["served_minimisations"] = served_minimisations(device)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C3")
    ap.add_argument("--precision", choices=["f64", "f32", "df64"], default="f64")
    ap.add_argument("--order", type=int, default=0, choices=(0, 1, 2),
                    help="internal node order: 0 as generated, 1 Morton, 2 reverse Cuthill-McKee")
    ap.add_argument("--flush-l2", action="store_true",
                    help="evict L2 before every timed step (automatic when a step's inputs are < 2 x L2)")
    ap.add_argument("--shuffle-nodes", action="store_true",
                    help="randomly permute the node ids (seed 4) before upload, to measure the node order")
    ap.add_argument("--sample-fraction", type=float, default=0.125)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-budget-gb", type=int, default=8)
    ap.add_argument("--minimize", action="store_true",
                    help="the full minimisation set: also the FP32, torch-memory and central-difference L-BFGS "
                         "runs and the paper's Benchmarks 4 and 6")
    ap.add_argument("--no-minimize", action="store_true", help="skip the minimisations")
    ap.add_argument("--paper-tables", action="store_true",
                    help="also time the energy and both gradients on the twisted bar, levels 1-5 (Tables 2 and 3)")
    ap.add_argument("--minimize-n", type=int, default=64)
    ap.add_argument("--minimize-iters", type=int, default=20000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
