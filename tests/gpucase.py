"""Shared set-up of GPU-vs-oracle comparisons: one case description builds both
the CUDA solver (through the C ABI binding) and the oracle configuration."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle
from paper_1909_13263_gb300 import inputs, native


@dataclass
class Case:
    dim: int
    nx: int
    ny: int
    ham: str
    bc: str = "periodic"
    weights: str = "arclength"
    alpha_mode: str = "global_lagged"
    precision: str = "fp64"
    lo: float = -1.0
    hi: float = 1.0
    dt_mode: str = "cfl"
    alpha_fixed: tuple = (0.0, 0.0)
    eps: float = 1e-6
    extra: dict = field(default_factory=dict)

    @property
    def dx(self):
        return inputs.axis(self.nx, self.lo, self.hi, self.bc)[1]

    @property
    def dy(self):
        return inputs.axis(self.ny, self.lo, self.hi, self.bc)[1] if self.dim == 2 else self.dx

    def solver(self, **kw):
        return native.Solver(dim=self.dim, nx=self.nx, ny=self.ny, bc=self.bc, xlo=self.lo, xhi=self.hi,
                             ylo=self.lo, yhi=self.hi, ham=self.ham, weights=self.weights, eps=self.eps,
                             dt_mode=self.dt_mode, alpha_mode=self.alpha_mode, alpha_fixed=self.alpha_fixed,
                             precision=self.precision, **kw)

    def cfg(self):
        am = self.alpha_mode
        if am == "default":
            am = "local_lagged" if self.dim == 1 else "global_lagged"
        return oracle.make_cfg(dim=self.dim, nx=self.nx, ny=self.ny, bc=self.bc, dx=self.dx, dy=self.dy,
                               ham=self.ham, weights=self.weights, eps=self.eps, dt_mode=self.dt_mode,
                               alpha_mode=am, alpha_fixed=self.alpha_fixed, xlo=self.lo,
                               ylo=self.lo if self.dim == 2 else 0.0)

    def field(self, seed=0, kind="rough"):
        if self.dim == 1:
            return inputs.random_field(1, self.nx, seed, kind)[0]
        return inputs.random_field(self.ny, self.nx, seed, kind)


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def oracle_stages(case: Case, phi0: np.ndarray, dt: float):
    """phi_1, phi_2, phi^{n+1} of one RK3 step with a given dt, alpha as the stage kernels use it.

    Flux alpha per mode: local (per node), fixed, or the grid maximum of the
    previous stage (lagged; the prime pass over phi0 for stage 1) or of the
    stage's own derivatives (exact)."""
    cfg = case.cfg()
    a_prev, _ = oracle.alpha_of(cfg, phi0)
    srcs = []
    L = []
    cur = phi0
    outs = []
    for s in range(3):
        a_own, _ = oracle.alpha_of(cfg, cur)
        if case.alpha_mode == "fixed":
            a_use = np.array(case.alpha_fixed)
        elif case.alpha_mode == "global_exact":
            a_use = a_own
        else:
            a_use = a_prev
        Ls = oracle.L_of(cfg, cur, a_use)
        if s == 0:
            nxt = phi0 + dt * Ls
        elif s == 1:
            nxt = 0.75 * phi0 + 0.25 * (cur + dt * Ls)
        else:
            nxt = phi0 / 3.0 + 2.0 * (cur + dt * Ls) / 3.0
        srcs.append(cur)
        L.append(Ls)
        outs.append(nxt)
        a_prev = a_own
        cur = nxt
    return outs


def oracle_steps(case: Case, phi0: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """nsteps RK3 steps (Step 5) of fixed size dt by the oracle, with the flux alpha as the stage
    kernels use it and the lagged alpha carried from step to step: a prime pass over phi0, then every
    stage's grid maximum serves the next stage (local modes use the node's own alpha, fixed the given
    pair, global exact the stage's own maximum)."""
    cfg = case.cfg()
    a_prev, _ = oracle.alpha_of(cfg, phi0)
    phi = np.array(phi0, dtype=np.float64)
    for _ in range(nsteps):
        cur = phi
        for s in range(3):
            a_own, _ = oracle.alpha_of(cfg, cur)
            if case.alpha_mode == "fixed":
                a_use = np.array(case.alpha_fixed)
            elif case.alpha_mode == "global_exact":
                a_use = a_own
            else:
                a_use = a_prev
            Ls = oracle.L_of(cfg, cur, a_use)
            if s == 0:
                cur = phi + dt * Ls
            elif s == 1:
                cur = 0.75 * phi + 0.25 * (cur + dt * Ls)
            else:
                cur = phi / 3.0 + 2.0 * (cur + dt * Ls) / 3.0
            a_prev = a_own
        phi = cur
    return phi
