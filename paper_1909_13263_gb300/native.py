"""Python binding of the C ABI in ``include/alweno.h`` (argument marshalling only).

Every step of the scheme runs in the CUDA library ``_build/libalweno.so``;
this module only converts arguments.  There is no CPU fallback: if the library
is missing or no CUDA device is present, calls raise ``AlwError``.

PyTorch is used for device memory (the library's allocator hook is pointed at
the torch caching allocator) and for streams (a solver enqueues its work on a
torch stream).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libalweno.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "alweno.h")

# enumerations (values as in include/alweno.h)
OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EBUSY, EBUDGET, ENOTFOUND = range(9)
STATUS = {0: "ALW_OK", 1: "ALW_EINVAL", 2: "ALW_ENOMEM", 3: "ALW_ECUDA", 4: "ALW_ENONFINITE",
          5: "ALW_ETIMEOUT", 6: "ALW_EBUSY", 7: "ALW_EBUDGET", 8: "ALW_ENOTFOUND"}
BC = {"periodic": 0, "linextrap": 1}
HAM = {"burgers2d": 0, "negcos2d": 1, "sin2d": 2, "advect1d": 3, "burgers1d": 4, "negcos1d": 5,
       "eikonal2d": 6, "nonconvex1d": 7, "optctrl2d": 8}
HAM_DIM = {"burgers2d": 2, "negcos2d": 2, "sin2d": 2, "eikonal2d": 2, "optctrl2d": 2, "advect1d": 1, "burgers1d": 1,
           "negcos1d": 1, "nonconvex1d": 1}
WEIGHTS = {"arclength": 0, "jp": 1}
ALPHA = {"default": -1, "local_lagged": 0, "local_exact": 1, "global_lagged": 2, "global_exact": 3,
         "fixed": 4}
DT = {"cfl": 0, "dx53": 1}
PREC = {"fp64": 0, "fp32": 1, "mixed": 2}


class AlwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("bc", ctypes.c_int32), ("xlo", ctypes.c_double), ("xhi", ctypes.c_double),
                ("ylo", ctypes.c_double), ("yhi", ctypes.c_double)]


class Hamiltonian(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("param", ctypes.c_double * 4)]


class Scheme(ctypes.Structure):
    _fields_ = [("weights", ctypes.c_int32), ("eps", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dt_mode", ctypes.c_int32), ("alpha_mode", ctypes.c_int32),
                ("alpha_fixed", ctypes.c_double * 2), ("precision", ctypes.c_int32)]


class State(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_int64), ("alpha", ctypes.c_double * 2)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("steps_per_graph", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("run", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("one_launch", ctypes.c_int32)]


ORDER = {"instance": 0, "largest_first": 1, "interleaved": 2}


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int64), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("rounds", ctypes.c_int64), ("arena_rows", ctypes.c_int64),
                ("free_rows", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def header_functions(path: str = HEADER):
    """Names of the functions declared in the C header."""
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:alw_status|const char \*)\s*(alw_\w+)\s*\(", text, re.M)))


def load():
    """Load the CUDA library (raises AlwError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise AlwError(ECUDA, f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        sig = {
            "alw_version": (ctypes.c_char_p, []),
            "alw_last_error": (ctypes.c_char_p, []),
            "alw_set_allocator": (ctypes.c_int, [ctypes.POINTER(Allocator)]),
            "alw_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Hamiltonian),
                                          ctypes.POINTER(Scheme), P, ctypes.POINTER(P)]),
            "alw_destroy": (ctypes.c_int, [P]),
            "alw_set_phi0": (ctypes.c_int, [P, P, SZ]),
            "alw_set_phi0_device": (ctypes.c_int, [P, P, I32, SZ]),
            "alw_step_to": (ctypes.c_int, [P, D, ctypes.POINTER(I64)]),
            "alw_advance": (ctypes.c_int, [P, I64]),
            "alw_run_stage": (ctypes.c_int, [P, I32, D]),
            "alw_sync": (ctypes.c_int, [P]),
            "alw_get_phi": (ctypes.c_int, [P, P, SZ]),
            "alw_get_phi_device": (ctypes.c_int, [P, P, I32, SZ]),
            "alw_get_stage_phi": (ctypes.c_int, [P, I32, P, SZ]),
            "alw_get_state": (ctypes.c_int, [P, ctypes.POINTER(State)]),
            "alw_set_state": (ctypes.c_int, [P, ctypes.POINTER(State), P, SZ]),
            "alw_memory_bytes": (ctypes.c_int, [P, ctypes.POINTER(SZ)]),
            "alw_step_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Hamiltonian),
                                                ctypes.POINTER(Scheme), P, P, D, I32, P]),
            "alw_batch_create": (ctypes.c_int, [ctypes.POINTER(Scheme), P, ctypes.POINTER(P)]),
            "alw_batch_add": (ctypes.c_int, [P, ctypes.POINTER(Grid), ctypes.POINTER(Hamiltonian), P, SZ, D,
                                             ctypes.POINTER(I32)]),
            "alw_batch_set_tuning": (ctypes.c_int, [P, ctypes.POINTER(BatchTuning)]),
            "alw_batch_get_tuning": (ctypes.c_int, [P, ctypes.POINTER(BatchTuning)]),
            "alw_batch_build": (ctypes.c_int, [P]),
            "alw_batch_run": (ctypes.c_int, [P, ctypes.POINTER(I64)]),
            "alw_batch_get_phi": (ctypes.c_int, [P, I32, P, SZ]),
            "alw_batch_get_state": (ctypes.c_int, [P, I32, ctypes.POINTER(State)]),
            "alw_batch_memory_bytes": (ctypes.c_int, [P, ctypes.POINTER(SZ)]),
            "alw_batch_destroy": (ctypes.c_int, [P]),
            "alw_server_create": (ctypes.c_int, [ctypes.POINTER(Scheme), SZ, I32, I32, P, ctypes.POINTER(P)]),
            "alw_server_set_round_steps": (ctypes.c_int, [P, I32]),
            "alw_server_set_round_tiles": (ctypes.c_int, [P, I32]),
            "alw_server_submit": (ctypes.c_int, [P, ctypes.POINTER(Grid), ctypes.POINTER(Hamiltonian), P, SZ, D,
                                                 ctypes.POINTER(ctypes.c_uint64)]),
            "alw_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, D, ctypes.POINTER(I32), P, SZ,
                                               ctypes.POINTER(RequestInfo)]),
            "alw_server_stats_get": (ctypes.c_int, [P, ctypes.POINTER(ServerStats)]),
            "alw_server_destroy": (ctypes.c_int, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def last_error() -> str:
    return load().alw_last_error().decode()


def check(st: int):
    if st != OK:
        raise AlwError(st, last_error())


# ---------------------------------------------------------------- allocator

_torch_alloc_keep = None


def use_torch_allocator(enable: bool = True):
    """Point the library's device allocations at the torch caching allocator."""
    global _torch_alloc_keep
    L = load()
    if not enable:
        check(L.alw_set_allocator(None))
        _torch_alloc_keep = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0))
        except Exception:  # out of memory -> NULL -> ALW_ENOMEM
            return None

    def _free(ptr, nbytes, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    a = Allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    _torch_alloc_keep = a
    check(L.alw_set_allocator(ctypes.byref(a)))


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------- solver

def _host_out(out, shape) -> np.ndarray:
    """A new float64 array of `shape`, or the caller's array after checking that it can take the result."""
    if out is None:
        return np.empty(shape, dtype=np.float64)
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.flags.writeable and out.shape == tuple(shape)):
        raise ValueError(f"out must be a writeable C-contiguous float64 array of shape {tuple(shape)}")
    return out


class Solver:
    """One HJ problem on the GPU (alw_create ... alw_destroy)."""

    def __init__(self, *, dim: int, nx: int, ny: int = 1, bc: str = "periodic", xlo: float, xhi: float,
                 ylo: float = 0.0, yhi: float = 1.0, ham: str, weights: str = "arclength", eps: float = 1e-6,
                 cfl: float = 0.6, dt_mode: str = "cfl", alpha_mode: str = "default",
                 alpha_fixed=(0.0, 0.0), precision: str = "fp64", stream=None):
        self._L = load()
        self.grid = Grid(dim, nx, ny if dim == 2 else 1, BC[bc], xlo, xhi, ylo, yhi)
        self.ham = Hamiltonian(HAM[ham], (ctypes.c_double * 4)(0, 0, 0, 0))
        self.scheme = Scheme(WEIGHTS[weights], eps, cfl, DT[dt_mode], ALPHA[alpha_mode],
                             (ctypes.c_double * 2)(*alpha_fixed), PREC[precision])
        self.nx, self.ny = nx, (ny if dim == 2 else 1)
        self.shape = (self.ny, self.nx) if dim == 2 else (self.nx,)
        h = ctypes.c_void_p()
        check(self._L.alw_create(ctypes.byref(self.grid), ctypes.byref(self.ham), ctypes.byref(self.scheme),
                                 ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h)))
        self._h = h

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def close(self):
        if getattr(self, "_h", None):
            self._L.alw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_phi0(self, phi0):
        """phi0: numpy array (host) or a CUDA torch tensor (float64/float32) of the grid's shape."""
        if hasattr(phi0, "is_cuda") and phi0.is_cuda:
            t = phi0.contiguous()
            if t.numel() != self.n:
                raise AlwError(EINVAL, f"expected {self.n} values, got {t.numel()}")
            dtype = {"torch.float64": 0, "torch.float32": 1}[str(t.dtype)]
            check(self._L.alw_set_phi0_device(self._h, ctypes.c_void_p(t.data_ptr()), dtype, t.numel()))
            return
        a = np.ascontiguousarray(phi0, dtype=np.float64)
        check(self._L.alw_set_phi0(self._h, a.ctypes.data, a.size))

    def step_to(self, t_final: float) -> int:
        n = ctypes.c_int64()
        check(self._L.alw_step_to(self._h, float(t_final), ctypes.byref(n)))
        return n.value

    def advance(self, nsteps: int):
        check(self._L.alw_advance(self._h, int(nsteps)))

    def run_stage(self, stage: int, dt: float):
        check(self._L.alw_run_stage(self._h, int(stage), float(dt)))

    def sync(self):
        check(self._L.alw_sync(self._h))

    def get_phi(self, out=None) -> np.ndarray:
        """phi on the host; into `out` (a C-contiguous float64 array of the grid's shape) when given."""
        out = _host_out(out, self.shape)
        check(self._L.alw_get_phi(self._h, out.ctypes.data, out.size))
        return out

    def get_phi_device(self, out):
        """Fill a contiguous CUDA torch tensor (float64 or float32) with phi."""
        dtype = {"torch.float64": 0, "torch.float32": 1}[str(out.dtype)]
        check(self._L.alw_get_phi_device(self._h, ctypes.c_void_p(out.data_ptr()), dtype, out.numel()))
        return out

    def get_stage_phi(self, stage: int) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        check(self._L.alw_get_stage_phi(self._h, int(stage), out.ctypes.data, out.size))
        return out

    def get_state(self) -> State:
        st = State()
        check(self._L.alw_get_state(self._h, ctypes.byref(st)))
        return st

    def set_state(self, state: State, phi):
        a = np.ascontiguousarray(phi, dtype=np.float64)
        check(self._L.alw_set_state(self._h, ctypes.byref(state), a.ctypes.data, a.size))

    def memory_bytes(self) -> int:
        b = ctypes.c_size_t()
        check(self._L.alw_memory_bytes(self._h, ctypes.byref(b)))
        return b.value


def step_noalloc(phi_in, phi_out, *, dim: int, nx: int, ny: int = 1, bc: str = "periodic", xlo: float, xhi: float,
                 ylo: float = 0.0, yhi: float = 1.0, ham: str, weights: str = "arclength", eps: float = 1e-6,
                 alpha_mode: str = "default", alpha_fixed=(0.0, 0.0), dt: float, nsteps: int = 1, stream=None):
    """alw_step_noalloc: nsteps FP64 RK3 steps of fixed dt on caller-owned CUDA float64 tensors,
    using the library's fixed working storage instead of allocating device memory."""
    import torch

    L = load()
    for t in (phi_in, phi_out):
        if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous() and t.numel() == nx * ny):
            raise AlwError(EINVAL, "phi_in/phi_out must be contiguous CUDA float64 tensors of nx*ny values")
        # the library works on the current device: its kernels there must not address another GPU's memory
        if t.device.index != torch.cuda.current_device():
            raise AlwError(EINVAL, f"tensor on cuda:{t.device.index}, but the current device is "
                                   f"cuda:{torch.cuda.current_device()}")
    g = Grid(dim, nx, ny if dim == 2 else 1, BC[bc], xlo, xhi, ylo, yhi)
    h = Hamiltonian(HAM[ham], (ctypes.c_double * 4)(0, 0, 0, 0))
    s = Scheme(WEIGHTS[weights], eps, 0.6, DT["cfl"], ALPHA[alpha_mode], (ctypes.c_double * 2)(*alpha_fixed),
               PREC["fp64"])
    check(L.alw_step_noalloc(ctypes.byref(g), ctypes.byref(h), ctypes.byref(s), ctypes.c_void_p(phi_in.data_ptr()),
                             ctypes.c_void_p(phi_out.data_ptr()), float(dt), int(nsteps),
                             ctypes.c_void_p(_stream_handle(stream))))
    return phi_out


class Batch:
    """Many independent 2D periodic instances advanced together (alw_batch_*)."""

    def __init__(self, *, weights: str = "arclength", precision: str = "mixed", eps: float = 1e-6, cfl: float = 0.6,
                 dt_mode: str = "cfl", alpha_mode: str = "default", alpha_fixed=(0.0, 0.0), stream=None):
        self._L = load()
        self.scheme = Scheme(WEIGHTS[weights], eps, cfl, DT[dt_mode], ALPHA[alpha_mode],
                             (ctypes.c_double * 2)(*alpha_fixed), PREC[precision])
        h = ctypes.c_void_p()
        check(self._L.alw_batch_create(ctypes.byref(self.scheme), ctypes.c_void_p(_stream_handle(stream)),
                                       ctypes.byref(h)))
        self._h = h
        self.shapes = []

    def add(self, *, nx: int, ny: int, xlo: float, xhi: float, ylo: float, yhi: float, ham: str, phi0,
            t_final: float) -> int:
        g = Grid(2, nx, ny, BC["periodic"], xlo, xhi, ylo, yhi)
        hm = Hamiltonian(HAM[ham], (ctypes.c_double * 4)(0, 0, 0, 0))
        a = np.ascontiguousarray(phi0, dtype=np.float64)
        i = ctypes.c_int32()
        check(self._L.alw_batch_add(self._h, ctypes.byref(g), ctypes.byref(hm), a.ctypes.data, a.size,
                                    float(t_final), ctypes.byref(i)))
        self.shapes.append((ny, nx))
        return i.value

    def set_tuning(self, order: str = None, steps_per_graph: int = 4, grid_ctas: int = 0, run: int = 4,
                   tile_w: int = 64, one_launch: bool = False):
        if order is None:
            check(self._L.alw_batch_set_tuning(self._h, None))
            return
        t = BatchTuning(ORDER[order], steps_per_graph, grid_ctas, run, tile_w, int(bool(one_launch)))
        check(self._L.alw_batch_set_tuning(self._h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = BatchTuning()
        check(self._L.alw_batch_get_tuning(self._h, ctypes.byref(t)))
        inv = {v: k for k, v in ORDER.items()}
        return {"order": inv.get(t.order, t.order), "steps_per_graph": t.steps_per_graph, "grid_ctas": t.grid_ctas,
                "run": t.run, "tile": f"{t.tile_w or 64}x32",
                "launches_per_stage": "one" if t.one_launch else "one per Hamiltonian"}

    def build(self):
        """Upload the instances and tune the work list now (run() does it on first use)."""
        check(self._L.alw_batch_build(self._h))

    def run(self) -> int:
        r = ctypes.c_int64()
        check(self._L.alw_batch_run(self._h, ctypes.byref(r)))
        return r.value

    def get_phi(self, i: int, out=None) -> np.ndarray:
        """phi of instance i on the host; into `out` (C-contiguous float64, the instance's shape) when given."""
        out = _host_out(out, self.shapes[i])
        check(self._L.alw_batch_get_phi(self._h, int(i), out.ctypes.data, out.size))
        return out

    def get_state(self, i: int) -> State:
        st = State()
        check(self._L.alw_batch_get_state(self._h, int(i), ctypes.byref(st)))
        return st

    def memory_bytes(self) -> int:
        b = ctypes.c_size_t()
        check(self._L.alw_batch_memory_bytes(self._h, ctypes.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.alw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request loop (alw_server_*)."""

    def __init__(self, *, hbm_budget_bytes: int, max_slots: int = 256, max_side: int = 2048,
                 weights: str = "arclength", precision: str = "mixed", eps: float = 1e-6, cfl: float = 0.6,
                 alpha_mode: str = "default", stream=None):
        self._L = load()
        self.scheme = Scheme(WEIGHTS[weights], eps, cfl, DT["cfl"], ALPHA[alpha_mode], (ctypes.c_double * 2)(0, 0),
                             PREC[precision])
        h = ctypes.c_void_p()
        check(self._L.alw_server_create(ctypes.byref(self.scheme), int(hbm_budget_bytes), int(max_slots),
                                        int(max_side), ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(h)))
        self._h = h
        self.shapes = {}

    def set_round_steps(self, steps: int):
        check(self._L.alw_server_set_round_steps(self._h, int(steps)))

    def set_round_tiles(self, tiles: int):
        check(self._L.alw_server_set_round_tiles(self._h, int(tiles)))

    def submit(self, *, nx: int, ny: int, xlo: float, xhi: float, ylo: float, yhi: float, ham: str, phi0,
               t_final: float) -> int:
        g = Grid(2, nx, ny, BC["periodic"], xlo, xhi, ylo, yhi)
        hm = Hamiltonian(HAM[ham], (ctypes.c_double * 4)(0, 0, 0, 0))
        a = np.ascontiguousarray(phi0, dtype=np.float64)
        rid = ctypes.c_uint64()
        check(self._L.alw_server_submit(self._h, ctypes.byref(g), ctypes.byref(hm), a.ctypes.data, a.size,
                                        float(t_final), ctypes.byref(rid)))
        self.shapes[rid.value] = (ny, nx)
        return rid.value

    def poll(self, rid: int, timeout: float = 0.0, fetch: bool = True):
        """(done, info dict, result or None); with fetch the result is copied out and the request forgotten."""
        done = ctypes.c_int32()
        info = RequestInfo()
        out = np.empty(self.shapes[rid], dtype=np.float64) if fetch else None
        check(self._L.alw_server_poll(self._h, ctypes.c_uint64(rid), float(timeout), ctypes.byref(done),
                                      out.ctypes.data if (fetch and out is not None) else None,
                                      out.size if fetch else 0, ctypes.byref(info)))
        if not done.value:
            return False, None, None
        d = {"status": info.status, "steps": info.steps, "queue_s": info.queue_s, "latency_s": info.latency_s}
        if fetch:
            self.shapes.pop(rid, None)
        return True, d, out

    def stats(self) -> dict:
        s = ServerStats()
        check(self._L.alw_server_stats_get(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._L.alw_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
