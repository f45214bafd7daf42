"""Python binding of libfemenergy.so (argument marshalling only).

The module-level functions carry the names of the C ABI in ``include/femenergy.h`` and take
plain integers for device pointers; :class:`FEMesh` wraps a context for torch tensors, and
:class:`EnergyFunction` is the ``torch.autograd.Function`` whose forward is the energy kernel
and whose backward is the exact-gradient kernel.  Every step of the evaluation runs in the
CUDA library; there is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library to load: FEMENERGY_LIBRARY names another build (e.g. libfemenergy_bounds.so)
LIB_PATH = os.environ.get("FEMENERGY_LIBRARY") or os.path.join(_HERE, "libfemenergy.so")

FE_OK, FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_EDOMAIN, FE_ETIMEOUT, FE_EBUSY = range(7)
FE_PLAPLACE, FE_NEOHOOKE, FE_PLAPLACE_LP = 0, 1, 2
FE_F64, FE_F32_COMP, FE_DF64 = 0, 1, 2
FE_ORDER_NONE, FE_ORDER_MORTON, FE_ORDER_RCM = 0, 1, 2
FE_INPUT_DEFORMATION, FE_INPUT_DISPLACEMENT = 0, 1
FE_VECTORS_CALLER, FE_VECTORS_DEVICE = 0, 1

_STATUS_NAMES = {0: "FE_OK", 1: "FE_EINVAL", 2: "FE_ENOMEM", 3: "FE_ECUDA", 4: "FE_EDOMAIN",
                 5: "FE_ETIMEOUT", 6: "FE_EBUSY"}


class FEError(RuntimeError):
    """A libfemenergy call returned a status other than FE_OK."""

    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double

# name -> argtypes (restype is int = fe_status unless listed in _RESTYPE)
_SIGNATURES = {
    "fe_version": [],
    "fe_last_error": [],
    "fe_node_order": [_int, _i64, _vp, _i64, _vp, _int, _vp],
    "fe_create": [_vp, _int, _vp],
    "fe_destroy": [_vp],
    "fe_set_stream": [_vp, _vp],
    "fe_mesh_upload": [_vp, _int, _int, _i64, _vp, _i64, _vp, _vp, _int],
    "fe_set_model": [_vp, _int, _dbl, _dbl, _dbl],
    "fe_set_load": [_vp, _vp],
    "fe_precompute": [_vp, ctypes.c_uint],
    "fe_set_precision": [_vp, _int],
    "fe_set_input": [_vp, _int],
    "fe_set_vector_order": [_vp, _int],
    "fe_to_device_order": [_vp, _vp, _vp],
    "fe_from_device_order": [_vp, _vp, _vp],
    "fe_footprint": [_vp, _vp],
    "fe_energy": [_vp, _vp, _vp, _vp],
    "fe_gradient_exact": [_vp, _vp, _vp],
    "fe_energy_gradient": [_vp, _vp, _vp, _vp],
    "fe_gradient_fd": [_vp, _vp, _dbl, _vp, _vp, _i64],
    "fe_hessian_vector": [_vp, _vp, _vp, _vp],
    "fe_cg_steihaug": [_vp, _vp, _vp, _dbl, _dbl, _int, _vp, _vp, _vp, _vp],
    "fe_lbfgs_create": [_vp, _int, _vp, _i64, _int],
    "fe_lbfgs_destroy": [_vp],
    "fe_lbfgs_reset": [_vp],
    "fe_lbfgs_pairs": [_vp, _vp],
    "fe_lbfgs_update": [_vp, _vp, _vp, _vp, _vp, _vp],
    "fe_lbfgs_direction": [_vp, _vp, _vp, _vp],
    "fe_lbfgs_step": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_energy_gradient_host": [_vp, _vp, _vp, _vp],
    "fe_energy_gradient_host_async": [_vp, _vp, _vp, _vp],
    "fe_host_wait": [_vp],
    "fe_sync_status": [_vp],
    "fe_set_wait_limit": [_vp, _i64],
    "fe_get_shape_gradients": [_vp, _vp, _vp],
    "fe_get_patches": [_vp, _vp, _vp],
    "fe_get_load_vector": [_vp, _vp],
    "fe_launch_count": [_vp, _vp],
    "fe_profile_enable": [_vp, _int],
    "fe_profile_read": [_vp, _vp, _vp, _int],
    "fe_diag_df64_log": [_vp, _vp, _vp, _i64],
    "fe_batch_work_bytes": [_vp, _vp],
    "fe_batch_create": [_vp, _int, _vp],
    "fe_batch_destroy": [_vp],
    "fe_batch_energy_gradient": [_vp, _vp, _int],
    "fe_batch_sync_status": [_vp],
    "fe_batch_launch_count": [_vp, _vp],
    "fe_batch_set_wait_limit": [_vp, _i64],
    "fe_fp64_rate": [_int, _int, _vp, _vp],
    "fe_debug_bounds_enabled": [],
    "fe_debug_bounds": [_int, _vp, _vp],
    "fe_debug_bounds_selftest": [_int, _i64, _i64],
    "fe_batch_plan": [_int, _vp, _vp, _i64, _vp, _vp, _vp, _vp],
    "fe_lbfgs_save": [_vp, _vp, _vp, _vp, _vp, _vp],
    "fe_lbfgs_restore": [_vp, _vp, _vp, _vp, _vp, _int],
    "fe_server_create": [_vp, _int, ctypes.c_size_t, _int],
    "fe_server_destroy": [_vp],
    "fe_server_submit": [_vp, _vp, _vp, _vp, _vp, _dbl, _vp],
    "fe_server_wait": [_vp, _i64, _vp, _vp, _vp],
    "fe_server_now": [_vp, _vp],
    "fe_server_stats": [_vp, _vp, _vp, _vp, _vp],
    "fe_server_reset_stats": [_vp],
    "fe_energy_noalloc": [_int, _vp, _int, _int, _int, _dbl, _dbl, _dbl, _i64, _vp, _i64, _vp, _vp,
                          _vp, _vp, _vp, _vp],
}
_RESTYPE = {"fe_version": ctypes.c_int, "fe_last_error": ctypes.c_char_p, "fe_debug_bounds_enabled": ctypes.c_int}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfemenergy.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_2109_01158_gb300.build` "
                "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, args in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = lib
    return _lib


def _call(name: str, *args) -> int:
    st = getattr(load_library(), name)(*args)
    if st != FE_OK:
        raise FEError(st, name, fe_last_error())
    return st


def _checked(name):
    def f(*args):
        return _call(name, *args)
    f.__name__ = name
    f.__doc__ = f"C ABI `{name}` (raises FEError on a status other than FE_OK)."
    return f


def fe_version() -> int:
    return load_library().fe_version()


def fe_last_error() -> str:
    msg = load_library().fe_last_error()
    return msg.decode() if msg else ""


fe_create = _checked("fe_create")
fe_destroy = _checked("fe_destroy")
fe_set_stream = _checked("fe_set_stream")
fe_mesh_upload = _checked("fe_mesh_upload")
fe_set_model = _checked("fe_set_model")
fe_set_load = _checked("fe_set_load")
fe_precompute = _checked("fe_precompute")
fe_set_precision = _checked("fe_set_precision")
fe_set_input = _checked("fe_set_input")
fe_set_vector_order = _checked("fe_set_vector_order")
fe_to_device_order = _checked("fe_to_device_order")
fe_from_device_order = _checked("fe_from_device_order")
fe_footprint = _checked("fe_footprint")
fe_node_order = _checked("fe_node_order")
fe_energy = _checked("fe_energy")
fe_gradient_exact = _checked("fe_gradient_exact")
fe_energy_gradient = _checked("fe_energy_gradient")
fe_gradient_fd = _checked("fe_gradient_fd")
fe_hessian_vector = _checked("fe_hessian_vector")
fe_cg_steihaug = _checked("fe_cg_steihaug")
fe_lbfgs_create = _checked("fe_lbfgs_create")
fe_lbfgs_destroy = _checked("fe_lbfgs_destroy")
fe_lbfgs_reset = _checked("fe_lbfgs_reset")
fe_lbfgs_pairs = _checked("fe_lbfgs_pairs")
fe_lbfgs_update = _checked("fe_lbfgs_update")
fe_lbfgs_direction = _checked("fe_lbfgs_direction")
fe_lbfgs_step = _checked("fe_lbfgs_step")


class LbfgsMemory:
    """The L-BFGS pairs of one minimisation on the device (fe_lbfgs): update(v_new, v, g_new, g)
    offers a pair and returns s.y (kept when > 0); direction(g) returns (d, g.d) with
    d = -H g of the limited-memory inverse Hessian."""

    def __init__(self, n: int, m: int = 10, device=0):
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.n, self.m = int(n), int(m)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            fe_lbfgs_create(ctypes.byref(h), self.device.index or 0, ctypes.c_void_p(stream), self.n, self.m)
        self.handle = h

    @staticmethod
    def device_bytes(n: int, m: int = 10) -> int:
        return 8 * 2 * (m + 1) * int(n)

    def _vec(self, x):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.numel() == self.n):
            raise TypeError(f"expected a float64 CUDA tensor of {self.n} entries")
        return x.contiguous()

    def reset(self):
        fe_lbfgs_reset(self.handle)

    def pairs(self) -> int:
        k = ctypes.c_int(0)
        fe_lbfgs_pairs(self.handle, ctypes.byref(k))
        return k.value

    def update(self, v_new, v, g_new, g) -> float:
        v_new, v, g_new, g = self._vec(v_new), self._vec(v), self._vec(g_new), self._vec(g)
        sy = ctypes.c_double(0.0)
        fe_lbfgs_update(self.handle, _ptr(v_new), _ptr(v), _ptr(g_new), _ptr(g), ctypes.byref(sy))
        return sy.value

    def direction(self, g, out=None):
        g = self._vec(g)
        d = out if out is not None else torch.empty_like(g)
        gd = ctypes.c_double(0.0)
        fe_lbfgs_direction(self.handle, _ptr(g), _ptr(d), ctypes.byref(gd))
        return d, gd.value

    def step(self, v_new, v, g_new, g, out=None):
        """update(v_new, v, g_new, g) and direction(g_new) in one host round trip: returns
        (d, s.y, g_new.d, max |g_new|)."""
        v_new, v, g_new, g = self._vec(v_new), self._vec(v), self._vec(g_new), self._vec(g)
        d = out if out is not None else torch.empty_like(g)
        o = (ctypes.c_double * 3)()
        fe_lbfgs_step(self.handle, _ptr(v_new), _ptr(v), _ptr(g_new), _ptr(g), _ptr(d), o)
        return d, o[0], o[1], o[2]

    def save(self):
        """(S, Y, SY, YY): the pairs in use, oldest first, as host arrays (k x n each) and their
        products s_i.y_j, y_i.y_j (k x k), for restore()."""
        S = np.empty((self.m, self.n)); Y = np.empty((self.m, self.n))
        SY = np.empty((self.m, self.m)); YY = np.empty((self.m, self.m))
        k = ctypes.c_int(0)
        fe_lbfgs_save(self.handle, _ptr(S), _ptr(Y), _ptr(SY), _ptr(YY), ctypes.byref(k))
        k = k.value
        return (S[:k].copy(), Y[:k].copy(), SY.ravel()[:k * k].reshape(k, k).copy(),
                YY.ravel()[:k * k].reshape(k, k).copy())

    def restore(self, state):
        """Replace the memory by a state from save() (same n, at most m pairs)."""
        S, Y, SY, YY = (np.ascontiguousarray(a, dtype=np.float64) for a in state)
        k = S.shape[0]
        if Y.shape[0] != k or S.shape[1:] != (self.n,) or Y.shape[1:] != (self.n,) or SY.shape != (k, k) \
                or YY.shape != (k, k):
            raise ValueError("state does not match this memory")
        fe_lbfgs_restore(self.handle, _ptr(S), _ptr(Y), _ptr(SY), _ptr(YY), int(k))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            fe_lbfgs_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
fe_energy_gradient_host = _checked("fe_energy_gradient_host")
fe_energy_gradient_host_async = _checked("fe_energy_gradient_host_async")
fe_get_shape_gradients = _checked("fe_get_shape_gradients")
fe_get_patches = _checked("fe_get_patches")
fe_get_load_vector = _checked("fe_get_load_vector")
fe_launch_count = _checked("fe_launch_count")
fe_profile_enable = _checked("fe_profile_enable")
fe_profile_read = _checked("fe_profile_read")
fe_energy_noalloc = _checked("fe_energy_noalloc")
fe_set_wait_limit = _checked("fe_set_wait_limit")
fe_diag_df64_log = _checked("fe_diag_df64_log")
fe_batch_work_bytes = _checked("fe_batch_work_bytes")
fe_batch_create = _checked("fe_batch_create")
fe_batch_destroy = _checked("fe_batch_destroy")
fe_batch_energy_gradient = _checked("fe_batch_energy_gradient")
fe_batch_launch_count = _checked("fe_batch_launch_count")
fe_batch_set_wait_limit = _checked("fe_batch_set_wait_limit")
fe_fp64_rate = _checked("fe_fp64_rate")
fe_debug_bounds = _checked("fe_debug_bounds")
fe_debug_bounds_selftest = _checked("fe_debug_bounds_selftest")
fe_batch_plan = _checked("fe_batch_plan")
fe_lbfgs_save = _checked("fe_lbfgs_save")
fe_lbfgs_restore = _checked("fe_lbfgs_restore")


def batch_plan(prep_tiles, elem_tiles, resident_blocks):
    """The batched kernel's work list: a list of (start, request, step) and the item count."""
    n = len(prep_tiles)
    pt = (ctypes.c_int64 * max(n, 1))(*prep_tiles)
    et = (ctypes.c_int64 * max(n, 1))(*elem_tiles)
    st = (ctypes.c_int64 * max(3 * n, 1))()
    rq = (ctypes.c_int32 * max(3 * n, 1))()
    sp = (ctypes.c_int32 * max(3 * n, 1))()
    tot = ctypes.c_int64()
    fe_batch_plan(n, pt, et, int(resident_blocks), st, rq, sp, ctypes.byref(tot))
    return [(st[q], rq[q], sp[q]) for q in range(3 * n)], tot.value
FE_RATE_DFMA, FE_RATE_DADD, FE_RATE_DMUL = range(3)


def fe_debug_bounds_enabled() -> int:
    return load_library().fe_debug_bounds_enabled()


def debug_bounds_enabled():
    """True when the loaded library is the bounds-checking build."""
    return bool(fe_debug_bounds_enabled())


def debug_bounds(device=0):
    """(site, index) of the first out-of-range index the kernels met since the last call, and
    clear it; (0, 0) when there was none (always in the ordinary build)."""
    site, index = ctypes.c_int(), ctypes.c_int64()
    fe_debug_bounds(int(device), ctypes.byref(site), ctypes.byref(index))
    return site.value, index.value


def debug_bounds_selftest(index, n, device=0):
    """One checked read of entry `index` of a device buffer of n doubles (bounds-checking
    build only)."""
    fe_debug_bounds_selftest(int(device), int(index), int(n))


def fp64_rate(device=0, op=FE_RATE_DFMA):
    """(operations per SM clock per SM, SM GHz during the measurement) of one FP64 operation."""
    r, ghz = ctypes.c_double(), ctypes.c_double()
    fe_fp64_rate(int(device), int(op), ctypes.byref(r), ctypes.byref(ghz))
    return r.value, ghz.value


def fe_batch_sync_status(batch) -> int:
    """Returns FE_OK or FE_EDOMAIN; raises on other errors."""
    st = load_library().fe_batch_sync_status(batch)
    if st not in (FE_OK, FE_EDOMAIN):
        raise FEError(st, "fe_batch_sync_status", fe_last_error())
    return st


class BatchItem(ctypes.Structure):
    """ctypes mirror of fe_batch_item."""
    _fields_ = [("mesh", _vp), ("v", _vp), ("J", _vp), ("g", _vp), ("work", _vp), ("done", _vp)]


class Batch:
    """Batched executor (fe_batch) on one device and stream: `run(items)` enqueues one
    energy + gradient evaluation of every (mesh, v, J, g, work) item in one persistent
    launch."""

    def __init__(self, device=0):
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device).cuda_stream
            fe_batch_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream))
        self.handle = h

    @staticmethod
    def work_bytes(mesh) -> int:
        n = ctypes.c_size_t(0)
        fe_batch_work_bytes(mesh.ctx, ctypes.byref(n))
        return n.value

    def run(self, items):
        """items: list of (FEMesh, v, J, g, work) with device tensors; work is a uint8 tensor
        of at least work_bytes(mesh) bytes whose data pointer is 256-byte aligned."""
        arr = (BatchItem * max(len(items), 1))()
        for k, item in enumerate(items):
            mesh, v, J, g, work = item[:5]
            done = item[5].data_ptr() if len(item) > 5 and item[5] is not None else None
            arr[k] = BatchItem(mesh.ctx.value, v.data_ptr(), J.data_ptr(), g.data_ptr(), work.data_ptr(), done)
        fe_batch_energy_gradient(self.handle, arr, len(items))

    def set_wait_limit(self, cycles: int = 0):
        """SM clocks a tile waits for the tiles it depends on (0 = the default 2e9)."""
        fe_batch_set_wait_limit(self.handle, int(cycles))

    def sync_status(self) -> int:
        return fe_batch_sync_status(self.handle)

    def launch_count(self) -> int:
        n = ctypes.c_int64(0)
        fe_batch_launch_count(self.handle, ctypes.byref(n))
        return n.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            fe_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

fe_server_create = _checked("fe_server_create")
fe_server_destroy = _checked("fe_server_destroy")
fe_server_submit = _checked("fe_server_submit")
fe_server_now = _checked("fe_server_now")
fe_server_stats = _checked("fe_server_stats")
fe_server_reset_stats = _checked("fe_server_reset_stats")


def fe_server_wait(server, ticket, t_arrival, t_start, t_done) -> int:
    """Returns FE_OK or FE_EDOMAIN (the request's status); raises on other errors."""
    st = load_library().fe_server_wait(server, ticket, t_arrival, t_start, t_done)
    if st not in (FE_OK, FE_EDOMAIN):
        raise FEError(st, "fe_server_wait", fe_last_error())
    return st


class NativeServer:
    """Continuous-batching server (fe_server): energy + gradient requests on resident
    FE_DF64 meshes, host vectors in and host results out, served by the library's own worker
    and completion threads.  `submit` keeps references to the arrays until `wait`."""

    def __init__(self, device=0, hbm_budget=8 << 30, max_batch=256):
        h = ctypes.c_void_p()
        fe_server_create(ctypes.byref(h), int(device), int(hbm_budget), int(max_batch))
        self.handle = h
        self._keep = {}

    def now(self) -> float:
        t = ctypes.c_double()
        fe_server_now(self.handle, ctypes.byref(t))
        return t.value

    def submit(self, mesh, v, J, g, t_arrival=-1.0) -> int:
        """v, g: float64 numpy arrays of mesh.ndof entries (C order); J: float64 array of one
        entry.  t_arrival: arrival time on the server clock (< 0 = now)."""
        for a, n in ((v, mesh.ndof), (g, mesh.ndof), (J, 1)):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == n):
                raise TypeError("v, g and J must be C-contiguous float64 numpy arrays of the mesh's sizes")
        t = ctypes.c_int64()
        fe_server_submit(self.handle, mesh.ctx, v.ctypes.data, J.ctypes.data, g.ctypes.data, float(t_arrival),
                         ctypes.byref(t))
        self._keep[t.value] = (mesh, v, J, g)
        return t.value

    def wait(self, ticket):
        """(status, t_arrival, t_start, t_done); status FE_OK or FE_EDOMAIN, raises otherwise."""
        ta, ts, td = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        try:
            st = fe_server_wait(self.handle, int(ticket), ctypes.byref(ta), ctypes.byref(ts), ctypes.byref(td))
        finally:
            self._keep.pop(ticket, None)
        return st, ta.value, ts.value, td.value

    def reset_stats(self):
        fe_server_reset_stats(self.handle)

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        fe_server_stats(self.handle, *[ctypes.byref(x) for x in v])
        return dict(zip(("batches", "max_batch", "launches", "completed"), (x.value for x in v)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            fe_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FE_PROFILE_STAGES = 5
PROFILE_STAGE_NAMES = ("node_prep", "element", "gather", "fd_element", "fd_gather")


def fe_sync_status(ctx) -> int:
    """Returns FE_OK or FE_EDOMAIN; raises on other errors."""
    st = load_library().fe_sync_status(ctx)
    if st not in (FE_OK, FE_EDOMAIN):
        raise FEError(st, "fe_sync_status", fe_last_error())
    return st


def fe_host_wait(ctx) -> int:
    """Returns FE_OK or FE_EDOMAIN; raises on other errors."""
    st = load_library().fe_host_wait(ctx)
    if st not in (FE_OK, FE_EDOMAIN):
        raise FEError(st, "fe_host_wait", fe_last_error())
    return st


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return a.data_ptr()
    return a.ctypes.data


def node_order(coords, elems, order):
    """The node renumbering fe_mesh_upload applies for `order` (host only, no GPU):
    perm[new] = old as an int32 array.  coords: (n_nodes, dim) floats; elems:
    (n_elems, dim+1) node ids."""
    X = np.ascontiguousarray(coords, dtype=np.float64)
    E = np.ascontiguousarray(elems, dtype=np.int32)
    nn, dim = X.shape
    perm = np.empty(nn, dtype=np.int32)
    fe_node_order(int(dim), nn, _ptr(X), E.shape[0], _ptr(E), int(order), _ptr(perm))
    return perm


class FEMesh:
    """One resident mesh with its precompute on a CUDA device.

    Arguments mirror ``fe_mesh_upload`` / ``fe_set_model`` / ``fe_set_load`` /
    ``fe_precompute``; arrays are host numpy arrays in the paper's layout.
    """

    def __init__(self, dim, d, coords, elems, dirichlet=None, *, model, p=2.0, C1=0.0, D1=0.0,
                 f=None, device=0, order=FE_ORDER_NONE, precisions=(FE_F64,)):
        if not torch.cuda.is_available():
            raise RuntimeError("FEMesh needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.dim, self.d = int(dim), int(d)
        self._coords = np.ascontiguousarray(coords, dtype=np.float64)
        self._elems = np.ascontiguousarray(elems, dtype=np.int32)
        self.nn, self.ne = self._coords.shape[0], self._elems.shape[0]
        self.ndof = self.nn * self.d
        dirichlet = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
        self.dirichlet = dirichlet
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._stream = torch.cuda.current_stream(self.device).cuda_stream
            fe_create(ctypes.byref(h), device, ctypes.c_void_p(self._stream))
        self.ctx = h
        fe_mesh_upload(self.ctx, self.dim, self.d, self.nn, _ptr(self._coords), self.ne,
                       _ptr(self._elems), _ptr(dirichlet), int(order))
        fe_set_model(self.ctx, int(model), float(p), float(C1), float(D1))
        if f is not None:
            f = np.ascontiguousarray(f, dtype=np.float64)
            fe_set_load(self.ctx, _ptr(f))
        mask = 0
        for prec in precisions:
            mask |= 1 << int(prec)
        fe_precompute(self.ctx, mask)
        fe_set_precision(self.ctx, int(precisions[0]))
        self.precision = int(precisions[0])
        self.input = FE_INPUT_DEFORMATION

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.dim, w.d, w.coords, w.elems, w.dirichlet, model=w.model, p=w.p, C1=w.C1,
                   D1=w.D1, f=w.f, **kw)

    # -- plumbing ------------------------------------------------------------------------
    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            fe_set_stream(self.ctx, ctypes.c_void_p(s))
            self._stream = s

    def _vec(self, v):
        if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64):
            raise TypeError("v must be a float64 CUDA tensor")
        if v.numel() != self.ndof:
            raise ValueError(f"v has {v.numel()} entries, expected {self.ndof}")
        return v.contiguous()

    def set_precision(self, prec):
        fe_set_precision(self.ctx, int(prec))
        self.precision = int(prec)

    def set_vector_order(self, order):
        """FE_VECTORS_CALLER (default) or FE_VECTORS_DEVICE: the numbering of the dof vectors of
        the evaluation, Hessian-vector, CG and central-difference calls."""
        fe_set_vector_order(self.ctx, int(order))
        self.vector_order = int(order)

    def to_device_order(self, x, out=None):
        """A dof vector in the caller's numbering -> the device numbering."""
        x = self._vec(x)
        self._sync_stream()
        y = out if out is not None else torch.empty_like(x)
        fe_to_device_order(self.ctx, _ptr(x), _ptr(y))
        return y

    def from_device_order(self, y, out=None):
        """A dof vector in the device numbering -> the caller's numbering."""
        y = self._vec(y)
        self._sync_stream()
        x = out if out is not None else torch.empty_like(y)
        fe_from_device_order(self.ctx, _ptr(y), _ptr(x))
        return x

    def set_input(self, kind):
        """FE_INPUT_DEFORMATION (v = X + u, default) or FE_INPUT_DISPLACEMENT (v = u)."""
        fe_set_input(self.ctx, int(kind))
        self.input = int(kind)

    # -- evaluation ----------------------------------------------------------------------
    def energy(self, v, densities=False):
        v = self._vec(v)
        self._sync_stream()
        J = torch.empty((), dtype=torch.float64, device=self.device)
        dens = torch.empty(self.ne, dtype=torch.float64, device=self.device) if densities else None
        fe_energy(self.ctx, _ptr(v), _ptr(J), _ptr(dens))
        return (J, dens) if densities else J

    def gradient_exact(self, v, out=None):
        v = self._vec(v)
        self._sync_stream()
        g = out if out is not None else torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        fe_gradient_exact(self.ctx, _ptr(v), _ptr(g))
        return g

    def energy_gradient(self, v, J=None, g=None):
        v = self._vec(v)
        self._sync_stream()
        J = J if J is not None else torch.empty((), dtype=torch.float64, device=self.device)
        g = g if g is not None else torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        fe_energy_gradient(self.ctx, _ptr(v), _ptr(J), _ptr(g))
        return J, g

    def gradient_fd(self, v, eps, dofs=None):
        v = self._vec(v)
        self._sync_stream()
        if dofs is None:
            g = torch.empty(self.ndof, dtype=torch.float64, device=self.device)
            fe_gradient_fd(self.ctx, _ptr(v), float(eps), _ptr(g), None, 0)
        else:
            dofs = torch.as_tensor(dofs, dtype=torch.int64).to(self.device).contiguous()
            g = torch.empty(dofs.numel(), dtype=torch.float64, device=self.device)
            fe_gradient_fd(self.ctx, _ptr(v), float(eps), _ptr(g), _ptr(dofs), dofs.numel())
        return g

    def hessian_vector(self, v, w, out=None):
        """Hw = d/dt grad J(v + t w) at t = 0 on the free dofs (FP64)."""
        v, w = self._vec(v), self._vec(w)
        self._sync_stream()
        Hw = out if out is not None else torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        fe_hessian_vector(self.ctx, _ptr(v), _ptr(w), _ptr(Hw))
        return Hw

    def cg_steihaug(self, v, g, radius, tol, max_cg, z=None, Hz=None):
        """Steihaug's truncated CG on the device for min g.z + z.H(v) z / 2, ||z|| <= radius.
        Returns (z, Hz, iterations, hit_boundary)."""
        v, g = self._vec(v), self._vec(g)
        self._sync_stream()
        z = z if z is not None else torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        Hz = Hz if Hz is not None else torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        k, bnd = ctypes.c_int(0), ctypes.c_int(0)
        fe_cg_steihaug(self.ctx, _ptr(v), _ptr(g), float(radius), float(tol), int(max_cg), _ptr(z), _ptr(Hz),
                       ctypes.byref(k), ctypes.byref(bnd))
        return z, Hz, k.value, bool(bnd.value)

    def energy_gradient_host(self, v_host, g_host=None):
        """End-to-end call on host buffers (numpy float64; pinned memory is fastest)."""
        v_host = np.ascontiguousarray(v_host, dtype=np.float64) if isinstance(v_host, np.ndarray) else v_host
        J = ctypes.c_double(0.0)
        if g_host is None:
            g_host = np.empty(self.ndof, dtype=np.float64)
        st = load_library().fe_energy_gradient_host(self.ctx, _ptr(v_host), ctypes.byref(J), _ptr(g_host))
        if st not in (FE_OK, FE_EDOMAIN):
            raise FEError(st, "fe_energy_gradient_host", fe_last_error())
        return J.value, g_host, st

    def energy_gradient_host_async(self, v_host, J_host, g_host):
        """Pipelined end-to-end call (fe_energy_gradient_host_async): enqueues the evaluation
        of v_host with J and g copied back into J_host (one float64) and g_host (ndof
        float64), and returns at once.  Use page-locked arrays (e.g. a pinned torch tensor's
        .numpy()) for the copies to overlap; read the outputs after host_wait()."""
        for a, n in ((v_host, self.ndof), (J_host, 1), (g_host, self.ndof)):
            if a.dtype != np.float64 or a.size < n or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffers must be C-contiguous float64 of the mesh's size")
        fe_energy_gradient_host_async(self.ctx, _ptr(v_host), _ptr(J_host), _ptr(g_host))

    def host_wait(self) -> int:
        """Wait for the pipelined evaluations; FE_OK or FE_EDOMAIN (raises on other errors)."""
        return fe_host_wait(self.ctx)

    def sync_status(self) -> int:
        return fe_sync_status(self.ctx)

    def set_wait_limit(self, cycles: int = 0):
        """SM clocks a kernel waits for a bulk copy before it reports FE_ETIMEOUT (0 = default)."""
        fe_set_wait_limit(self.ctx, int(cycles))

    # -- inspection ----------------------------------------------------------------------
    def shape_gradients(self):
        dphi = np.empty(self.ne * (self.dim + 1) * self.dim)
        vol = np.empty(self.ne)
        fe_get_shape_gradients(self.ctx, _ptr(dphi), _ptr(vol))
        return dphi, vol

    def patches(self):
        row_ptr = np.empty(self.nn + 1, dtype=np.int64)
        ent = np.empty(max(self.ne * (self.dim + 1), 1), dtype=np.int64)
        fe_get_patches(self.ctx, _ptr(row_ptr), _ptr(ent))
        return row_ptr, ent[: self.ne * (self.dim + 1)]

    def load_vector(self):
        b = np.empty(self.ndof)
        fe_get_load_vector(self.ctx, _ptr(b))
        return b

    def diag_df64_log(self, x):
        """log(x) by the double-float logarithm of the FE_DF64 kernels (diagnostic)."""
        x = torch.as_tensor(x, dtype=torch.float64).to(self.device).contiguous()
        y = torch.empty_like(x)
        self._sync_stream()
        fe_diag_df64_log(self.ctx, _ptr(x), _ptr(y), x.numel())
        return y

    def footprint(self) -> int:
        n = ctypes.c_size_t(0)
        fe_footprint(self.ctx, ctypes.byref(n))
        return n.value

    def launch_count(self) -> int:
        n = ctypes.c_int64(0)
        fe_launch_count(self.ctx, ctypes.byref(n))
        return n.value

    def profile(self, enable: bool = True):
        fe_profile_enable(self.ctx, 1 if enable else 0)

    def profile_read(self):
        """{stage: (total ms, launches)} since the last read; synchronises the stream."""
        ms = np.zeros(FE_PROFILE_STAGES)
        n = np.zeros(FE_PROFILE_STAGES, dtype=np.int64)
        fe_profile_read(self.ctx, _ptr(ms), _ptr(n), FE_PROFILE_STAGES)
        return {PROFILE_STAGE_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(FE_PROFILE_STAGES)}

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            fe_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class EnergyFunction(torch.autograd.Function):
    """J = energy(v) with the exact-gradient kernel as its backward.

    The gradient is taken with respect to the free dofs: Dirichlet dofs are data of the
    problem and receive 0 (Remark 1 of the paper restricts the gradient to free dofs)."""

    @staticmethod
    def forward(ctx, v, mesh: FEMesh):
        ctx.mesh = mesh
        ctx.save_for_backward(v)
        return mesh.energy(v)

    @staticmethod
    def backward(ctx, grad_out):
        (v,) = ctx.saved_tensors
        g = ctx.mesh.gradient_exact(v)
        return grad_out * g, None


def energy(v, mesh: FEMesh):
    """Differentiable energy: ``energy(v, mesh).backward()`` runs the exact-gradient kernel."""
    return EnergyFunction.apply(v, mesh)
