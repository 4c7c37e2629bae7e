"""Exact solutions by characteristics, valid before characteristics cross.

For phi_t + H(phi_x) = 0 with phi0(x) = -cos(pi x): p = phi_x is constant
along x = x0 + H'(p0) t, p0 = pi sin(pi x0), and
phi(x, t) = phi0(x0) + t (p0 H'(p0) - H(p0)).
The 2D problems of Examples 3 and 4 reduce to these with xi = (x + y)/2:
phi(x, y, t) = w((x + y)/2, t) where w solves the 1D problem with the same H
applied to w_xi (since phi_x = phi_y = w_xi / 2 and H depends on phi_x + phi_y).
"""
from __future__ import annotations

import numpy as np

PI = np.pi

# (H, H', H'') of the 1D Hamiltonians used by the smooth examples
_H1 = {
    "advect1d": (lambda p: p, lambda p: np.ones_like(p), lambda p: np.zeros_like(p)),
    "burgers1d": (lambda p: 0.5 * (p + 1) ** 2, lambda p: p + 1, lambda p: np.ones_like(p)),
    "negcos1d": (lambda p: -np.cos(p + 1), lambda p: np.sin(p + 1), lambda p: np.cos(p + 1)),
}


def negcos_1d(ham: str, x, t: float, period: float = 2.0):
    """phi(x, t) for phi0 = -cos(pi x) on a periodic line of the given period."""
    H, H1, H2 = _H1[ham]
    x = np.asarray(x, dtype=np.float64)
    x0 = x.copy()
    for _ in range(100):
        p0 = PI * np.sin(PI * x0)
        g = x0 + H1(p0) * t - x
        dg = 1.0 + H2(p0) * PI * PI * np.cos(PI * x0) * t
        step = g / dg
        x0 = x0 - step
        if np.max(np.abs(step)) < 1e-15:
            break
    p0 = PI * np.sin(PI * x0)
    return -np.cos(PI * x0) + t * (p0 * H1(p0) - H(p0))


def negcos_diag_2d(ham2d: str, x, y, t: float):
    """phi(x, y, t) for phi0 = -cos(pi (x + y)/2), H = H1(phi_x + phi_y)."""
    ham1 = {"burgers2d": "burgers1d", "negcos2d": "negcos1d"}[ham2d]
    X, Y = np.meshgrid(x, y, indexing="xy")
    return negcos_1d(ham1, 0.5 * (X + Y), t)
