"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds grids, initial data and the seeded workload generators that
both the CUDA path and the CPU oracle are fed with.  It contains none of the
scheme's arithmetic (no differences, weights, fluxes or time stepping).

Grid convention: a periodic grid has ``n`` nodes on ``[lo, hi)`` with
``dx = (hi - lo) / n``; a linear-extrapolation grid has ``n`` nodes on
``[lo, hi]`` including both ends with ``dx = (hi - lo) / (n - 1)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED = 190913263


def axis(n: int, lo: float, hi: float, bc: str):
    """Node coordinates and spacing of one axis."""
    if bc == "periodic":
        dx = (hi - lo) / n
    elif bc == "linextrap":
        if n < 2:
            raise ValueError("a linear-extrapolation axis needs at least 2 nodes")
        dx = (hi - lo) / (n - 1)
    else:
        raise ValueError(bc)
    return lo + dx * np.arange(n, dtype=np.float64), dx


def phi0_negcos_1d(x):
    """phi0(x) = -cos(pi x)  (Examples 1, 2, 6, 7)."""
    return -np.cos(np.pi * x)


def phi0_negcos_diag_2d(x, y, theta: float = 0.0):
    """phi0(x, y) = -cos(pi (x + y) / 2 + theta)  (Examples 3, 4, 9; theta = phase shift)."""
    X, Y = np.meshgrid(x, y, indexing="xy")
    return -np.cos(np.pi * (X + Y) / 2.0 + theta)


def phi0_riemann_2d(x, y):
    """phi0(x, y) = pi (|y| - |x|)  (Example 10)."""
    X, Y = np.meshgrid(x, y, indexing="xy")
    return np.pi * (np.abs(Y) - np.abs(X))


def phi0_eikonal_2d(x, y):
    """phi0(x, y) = (cos(2 pi x) - 1)(cos(2 pi y) - 1)/4 - 1  (Example 12)."""
    X, Y = np.meshgrid(x, y, indexing="xy")
    return 0.25 * (np.cos(2 * np.pi * X) - 1.0) * (np.cos(2 * np.pi * Y) - 1.0) - 1.0


def phi0_corners_1d(x):
    """Example 5: phi(x, 0) = f(x - 0.5), f a linear ramp plus four smooth pieces meeting at
    corners (x = -1/3, 0, 1/3), extended periodically from [-1, 1).

    The third piece is taken as 15/2 - 3 cos(2 pi x): the printed constant 5/2 would leave
    jumps of 5 at x = 0 and x = 1/3, whereas 15/2 makes f continuous there and periodic."""
    z = np.asarray(x, dtype=np.float64) - 0.5
    z = (z + 1.0) % 2.0 - 1.0
    base = -(np.sqrt(3.0) / 2.0 + 4.5 + 2.0 * np.pi / 3.0) * (z + 1.0)
    out = np.where(z < -1.0 / 3.0, 2.0 * np.cos(1.5 * np.pi * z * z) - np.sqrt(3.0),
          np.where(z < 0.0, 1.5 + 3.0 * np.cos(2.0 * np.pi * z),
          np.where(z < 1.0 / 3.0, 7.5 - 3.0 * np.cos(2.0 * np.pi * z),
                   (28.0 + 4.0 * np.pi + np.cos(3.0 * np.pi * z)) / 3.0 + 6.0 * np.pi * z * (z - 1.0))))
    return base + out


def phi0_abs_1d(x):
    """Example 8: phi(x, 0) = -2|x|."""
    return -2.0 * np.abs(np.asarray(x, dtype=np.float64))


def random_field(ny: int, nx: int, seed: int, kind: str = "smooth") -> np.ndarray:
    """Seeded test data: 'smooth' (few Fourier modes), 'rough' (smooth + kinks + noise)."""
    rng = np.random.default_rng(seed)
    y = np.linspace(0.0, 1.0, ny, endpoint=False)[:, None]
    x = np.linspace(0.0, 1.0, nx, endpoint=False)[None, :]
    f = np.zeros((ny, nx))
    for _ in range(4):
        kx, ky = rng.integers(0, 4, size=2)
        a, ph = rng.normal(), rng.uniform(0, 2 * np.pi)
        f += a * np.cos(2 * np.pi * (kx * x + ky * y) + ph)
    if kind == "rough":
        f += 0.5 * np.abs(np.sin(3 * np.pi * (x - 0.3 * y)))
        f += 0.05 * rng.standard_normal((ny, nx))
    return f


# --- configurations of the paper's examples --------------------------------

@dataclass(frozen=True)
class Problem:
    name: str
    dim: int
    ham: str
    lo: float
    hi: float
    bc: str
    t_final: float
    phi0: str


PROBLEMS = {
    "ex1_advect": Problem("ex1_advect", 1, "advect1d", -1.0, 1.0, "periodic", 2.0, "negcos1d"),
    "ex2_negcos1d": Problem("ex2_negcos1d", 1, "negcos1d", -1.0, 1.0, "periodic", 0.5 / math.pi**2, "negcos1d"),
    "ex6_burgers1d_smooth": Problem("ex6_burgers1d_smooth", 1, "burgers1d", -1.0, 1.0, "periodic",
                                    0.5 / math.pi**2, "negcos1d"),
    "ex6_burgers1d_kink": Problem("ex6_burgers1d_kink", 1, "burgers1d", -1.0, 1.0, "periodic",
                                  3.5 / math.pi**2, "negcos1d"),
    "ex3_burgers2d": Problem("ex3_burgers2d", 2, "burgers2d", -2.0, 2.0, "periodic", 0.5 / math.pi**2, "negcos_diag"),
    "ex4_negcos2d": Problem("ex4_negcos2d", 2, "negcos2d", -2.0, 2.0, "periodic", 0.5 / math.pi**2, "negcos_diag"),
    "ex10_sin2d": Problem("ex10_sin2d", 2, "sin2d", -1.0, 1.0, "linextrap", 1.0, "riemann"),
    "ex12_eikonal2d": Problem("ex12_eikonal2d", 2, "eikonal2d", 0.0, 1.0, "periodic", 0.6, "eikonal"),
    "ex5_corners": Problem("ex5_corners", 1, "advect1d", -1.0, 1.0, "periodic", 2.0, "corners"),
    "ex8_nonconvex1d": Problem("ex8_nonconvex1d", 1, "nonconvex1d", -1.0, 1.0, "periodic", 1.0, "abs"),
    "ex11_optctrl2d": Problem("ex11_optctrl2d", 2, "optctrl2d", -math.pi, math.pi, "periodic", 1.0, "zero"),
}


def initial(problem: Problem, n: int, theta: float = 0.0):
    """(phi0, dx) for a problem on an n-node (or n x n) grid."""
    x, dx = axis(n, problem.lo, problem.hi, problem.bc)
    if problem.dim == 1:
        f = {"negcos1d": phi0_negcos_1d, "corners": phi0_corners_1d, "abs": phi0_abs_1d}[problem.phi0]
        return f(x), dx
    if problem.phi0 == "negcos_diag":
        return phi0_negcos_diag_2d(x, x, theta), dx
    if problem.phi0 == "riemann":
        return phi0_riemann_2d(x, x), dx
    if problem.phi0 == "eikonal":
        return phi0_eikonal_2d(x, x), dx
    if problem.phi0 == "zero":
        return np.zeros((n, n)), dx
    raise ValueError(problem.phi0)


# --- multi-instance workloads ------------------------------------------------

@dataclass(frozen=True)
class Instance:
    n: int            # nodes per side (square grid)
    ham: str          # "burgers2d" or "negcos2d"
    theta: float      # phase shift of phi0
    t_final: float


def batch_instances(count: int = 512, lo_side: int = 64, hi_side: int = 1024, seed: int = SEED):
    """Instances of the batched workload: log-uniform square grids, 50/50 Hamiltonians,
    random phase, t_final ~ U[0.1, 0.5]/pi^2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(lo_side), math.log(hi_side)))))
        h = "burgers2d" if rng.random() < 0.5 else "negcos2d"
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        tf = float(rng.uniform(0.1, 0.5) / math.pi**2)
        out.append(Instance(n, h, theta, tf))
    return out


def instance_phi0(inst: Instance):
    x, dx = axis(inst.n, -2.0, 2.0, "periodic")
    return phi0_negcos_diag_2d(x, x, inst.theta), dx


def request_stream(rate: float, count: int, lo_side: int = 128, hi_side: int = 2048, seed: int = SEED):
    """Poisson arrivals (seconds from start) with instances drawn like the batch mix."""
    rng = np.random.default_rng(seed + int(rate))
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps)
    inst = batch_instances(count, lo_side, hi_side, seed=seed + int(rate) + 1)
    return list(zip(arrivals.tolist(), inst))
