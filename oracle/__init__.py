"""FP64 CPU oracle for the arc-length WENO scheme (test infrastructure only).

The oracle is ``alw_oracle.c`` (plain C, double precision, no FMA
contraction), compiled here into ``_build/liboracle.so`` and called through
ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the timed CPU
baseline of ``bench.py`` may import this package; the product path never
does.  It shares no code with the CUDA library.

Enumerations below are the oracle's own; callers translate names such as
``"burgers2d"`` into them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

HAM = {"burgers2d": 0, "negcos2d": 1, "sin2d": 2, "advect1d": 3, "burgers1d": 4,
       "negcos1d": 5, "eikonal2d": 6, "nonconvex1d": 7,
       "optctrl2d": 8}
BC = {"periodic": 0, "linextrap": 1}
WEIGHTS = {"arclength": 0, "jp": 1}
ALPHA = {"local_lagged": 0, "local_exact": 1, "global_lagged": 2, "global_exact": 3, "fixed": 4}
DT = {"cfl": 0, "dx53": 1}


class OrcCfg(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("bc", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("ham", ctypes.c_int32), ("weights", ctypes.c_int32), ("eps", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt_mode", ctypes.c_int32), ("alpha_mode", ctypes.c_int32),
                ("alpha_fixed", ctypes.c_double * 2), ("xlo", ctypes.c_double), ("ylo", ctypes.c_double)]


L_FN = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction). Returns the .so path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_arclength.restype = ctypes.c_double
        L.orc_arclength.argtypes = [ctypes.c_double] * 4
        for name in ("orc_phix_minus", "orc_phix_plus"):
            f = getattr(L, name)
            f.restype = ctypes.c_double
            f.argtypes = [dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp, dp]
        L.orc_ham.restype = ctypes.c_int
        L.orc_ham.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [dp, dp, dp]
        L.orc_hhat.restype = ctypes.c_double
        L.orc_hhat.argtypes = [ctypes.c_int] + [ctypes.c_double] * 8
        cp = ctypes.POINTER(OrcCfg)
        L.orc_point_derivs.restype = None
        L.orc_point_derivs.argtypes = [cp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_derivs.restype = None
        L.orc_derivs.argtypes = [cp, dp, dp, dp, dp, dp]
        L.orc_alpha_max.restype = ctypes.c_int
        L.orc_alpha_max.argtypes = [cp, dp, dp, dp, dp, dp]
        L.orc_alpha_of.restype = ctypes.c_int
        L.orc_alpha_of.argtypes = [cp, dp, dp]
        L.orc_L_from_derivs.restype = None
        L.orc_L_from_derivs.argtypes = [cp, dp, dp, dp, dp, dp, dp]
        L.orc_solve.restype = ctypes.c_int
        L.orc_solve.argtypes = [cp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64, dp,
                                ctypes.POINTER(ctypes.c_int64), dp]
        L.orc_rk3_step_generic.restype = ctypes.c_int
        L.orc_rk3_step_generic.argtypes = [ctypes.c_int64, dp, ctypes.c_double, L_FN, ctypes.c_void_p]
        L.orc_point_L.restype = ctypes.c_double
        L.orc_point_L.argtypes = [cp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_node_alpha.restype = None
        L.orc_node_alpha.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 6 + [dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_cfg(*, dim, nx, ny=1, bc="periodic", dx, dy=None, ham, weights="arclength", eps=1e-6,
             cfl=0.6, dt_mode="cfl", alpha_mode="local_lagged", alpha_fixed=(0.0, 0.0),
             xlo=0.0, ylo=0.0) -> OrcCfg:
    c = OrcCfg()
    c.dim, c.nx, c.ny = dim, nx, (ny if dim == 2 else 1)
    c.bc = BC[bc]
    c.dx = dx
    c.dy = dx if dy is None else dy
    c.ham = HAM[ham]
    c.weights = WEIGHTS[weights]
    c.eps, c.cfl = eps, cfl
    c.dt_mode = DT[dt_mode]
    c.alpha_mode = ALPHA[alpha_mode]
    c.alpha_fixed[0], c.alpha_fixed[1] = alpha_fixed
    c.xlo, c.ylo = xlo, ylo
    return c


def arclength(b: float, c: float, z0: float, z1: float) -> float:
    return lib().orc_arclength(b, c, z0, z1)


def phix_minus(p6, dx, weights="arclength", eps=1e-6):
    """phi_x^- at x_i from phi_{i-3..i+2}; returns (value, candidates, betas, omegas)."""
    p = _f64(p6)
    assert p.shape == (6,)
    cand, beta, omega = np.zeros(3), np.zeros(3), np.zeros(3)
    v = lib().orc_phix_minus(_dp(p), dx, WEIGHTS[weights], eps, _dp(cand), _dp(beta), _dp(omega))
    return v, cand, beta, omega


def phix_plus(q6, dx, weights="arclength", eps=1e-6):
    """phi_x^+ at x_i from phi_{i-2..i+3}; returns (value, candidates, betas, omegas)."""
    q = _f64(q6)
    assert q.shape == (6,)
    cand, beta, omega = np.zeros(3), np.zeros(3), np.zeros(3)
    v = lib().orc_phix_plus(_dp(q), dx, WEIGHTS[weights], eps, _dp(cand), _dp(beta), _dp(omega))
    return v, cand, beta, omega


def ham(kind: str, p: float, q: float = 0.0, x: float = 0.0, y: float = 0.0):
    """(H, H_p, H_q) at the position (x, y) (only Example 11's H depends on it)."""
    H, Hp, Hq = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().orc_ham(HAM[kind], x, y, p, q, ctypes.byref(H), ctypes.byref(Hp), ctypes.byref(Hq))
    if st:
        raise ValueError(kind)
    return H.value, Hp.value, Hq.value


def node_alpha(kind: str, dim: int, um, up, vm=0.0, vp=0.0, x=0.0, y=0.0):
    """The node-local Lax-Friedrichs alpha pair (alpha_x, alpha_y) at the position (x, y)."""
    out = np.zeros(2)
    lib().orc_node_alpha(HAM[kind], dim, x, y, um, up, vm, vp, _dp(out))
    return out


def hhat(kind: str, up, um, vp=0.0, vm=0.0, ax=0.0, ay=0.0, x=0.0, y=0.0) -> float:
    return lib().orc_hhat(HAM[kind], x, y, up, um, vp, vm, ax, ay)


def derivs(cfg: OrcCfg, phi: np.ndarray):
    """(u^-, u^+, v^-, v^+) at every node of phi (shape (ny, nx) or (nx,))."""
    p = _f64(phi)
    outs = [np.zeros_like(p) for _ in range(4)]
    lib().orc_derivs(ctypes.byref(cfg), _dp(p), *[_dp(o) for o in outs])
    return tuple(outs)


def alpha_of(cfg: OrcCfg, phi: np.ndarray):
    p = _f64(phi)
    out = np.zeros(2)
    st = lib().orc_alpha_of(ctypes.byref(cfg), _dp(p), _dp(out))
    return out, st


def L_of(cfg: OrcCfg, phi: np.ndarray, alpha) -> np.ndarray:
    p = _f64(phi)
    um, up, vm, vp = derivs(cfg, p)
    a = _f64(alpha)
    L = np.zeros_like(p)
    lib().orc_L_from_derivs(ctypes.byref(cfg), _dp(um), _dp(up), _dp(vm), _dp(vp), _dp(a), _dp(L))
    return L


def point_L(cfg: OrcCfg, phi: np.ndarray, i: int, j: int, alpha) -> float:
    """L(phi) at one node; phi must be C-contiguous float64 (not copied if so)."""
    a = _f64(alpha)
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    return lib().orc_point_L(ctypes.byref(cfg), _dp(phi), i, j, _dp(a))


def point_derivs(cfg: OrcCfg, phi: np.ndarray, i: int, j: int) -> np.ndarray:
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    out = np.zeros(4)
    lib().orc_point_derivs(ctypes.byref(cfg), _dp(phi), i, j, _dp(out))
    return out


def solve(cfg: OrcCfg, phi0: np.ndarray, t_final: float, t0: float = 0.0, max_steps: int = 10**8,
          alpha_state=None):
    """Advance phi0 to t_final with TVD-RK3.  Returns (phi, steps, t, alpha_state, status)."""
    phi = _f64(phi0).copy()
    a = np.array([-1.0, -1.0]) if alpha_state is None else _f64(alpha_state).copy()
    steps = ctypes.c_int64()
    t = ctypes.c_double()
    st = lib().orc_solve(ctypes.byref(cfg), _dp(phi), t0, t_final, max_steps, _dp(a),
                         ctypes.byref(steps), ctypes.byref(t))
    return phi, steps.value, t.value, a, st


def rk3_step_generic(y0, dt: float, Lfun) -> np.ndarray:
    """One TVD-RK3 step of dy/dt = Lfun(y) with the oracle's stage combination."""
    y = _f64(y0).copy()

    def cb(n, yp, outp, ctx):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        oo = np.ctypeslib.as_array(outp, shape=(n,))
        oo[:] = Lfun(yy.copy())

    fn = L_FN(cb)
    st = lib().orc_rk3_step_generic(y.size, _dp(y), dt, fn, None)
    if st:
        raise MemoryError
    return y
