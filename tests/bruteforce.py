"""Independent brute-force restatement of the scheme for tiny inputs.

Written from the paper's definitions, not from the oracle: every candidate
polynomial is obtained by solving its cell-average conditions (Step 2, Step 1)
exactly in rational arithmetic, in the global coordinate; arc lengths
(Eq. length) are integrated by Gauss-Legendre quadrature.  The "+" side is
built left to right on the sub-stencils T_k^+ = {x_{i-2+k}, ..., x_{i+1+k}}
with the mirrored linear weights (3/10, 6/10, 1/10) and the smoothness
interval [x_i, x_{i+1}].  Slow; meant for a few dozen points.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

D_MINUS = (Fr(1, 10), Fr(6, 10), Fr(3, 10))
D_PLUS = (Fr(3, 10), Fr(6, 10), Fr(1, 10))


def solve_exact(A, b):
    """Gaussian elimination over the rationals."""
    n = len(b)
    M = [list(row) + [bb] for row, bb in zip(A, b)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return [M[r][n] / M[r][r] for r in range(n)]


def cell_average_poly(xs, avgs):
    """Coefficients a_0..a_m (p = sum a_m x^m, m = len(avgs)-1) with
    (1/(x_{j+1}-x_j)) int_{x_j}^{x_{j+1}} p = avgs[j]; xs has len(avgs)+1 nodes."""
    deg = len(avgs) - 1
    A = []
    for j in range(len(avgs)):
        a, b = xs[j], xs[j + 1]
        A.append([(b ** (m + 1) - a ** (m + 1)) / ((m + 1) * (b - a)) for m in range(deg + 1)])
    return solve_exact(A, list(avgs))


def peval(coef, x):
    return sum(c * x ** m for m, c in enumerate(coef))


def pderiv(coef):
    return [m * c for m, c in enumerate(coef)][1:]


_GL_X, _GL_W = np.polynomial.legendre.leggauss(20)


def arc_length_linear_slope(uL: float, uR: float, width: float) -> float:
    """int over an interval of width `width` of sqrt(1 + u(s)^2), u linear from uL to uR.

    Composite Gauss-Legendre in u: pieces no wider than 0.1 (1 + |u|) so each
    sees an integrand far from its complex singularities at u = +-i."""
    if uL == uR:
        return width * float(np.sqrt(1.0 + uL * uL))
    lo, hi = min(uL, uR), max(uL, uR)
    edges = [lo]
    while edges[-1] < hi:
        edges.append(min(hi, edges[-1] + 0.1 * (1.0 + abs(edges[-1]))))
    e = np.array(edges)
    a, b = e[:-1, None], e[1:, None]
    u = 0.5 * (b - a) * _GL_X[None, :] + 0.5 * (a + b)
    total = float(np.sum(0.5 * (b - a) * _GL_W[None, :] * np.sqrt(1.0 + u * u)))
    return width * total / (hi - lo)


def one_sided(phi_vals, x_vals, i, side: str, weights: str, eps: float):
    """phi_x^- (side '-') or phi_x^+ (side '+') at local index i of the arrays.

    phi_vals, x_vals: sequences of Fractions long enough to hold i-3..i+3.
    Returns (value, candidates, betas, omegas) as floats.
    """
    dx = x_vals[i] - x_vals[i - 1]
    dplus = [(phi_vals[j + 1] - phi_vals[j]) / dx for j in range(len(phi_vals) - 1)]
    cands, betas = [], []
    for k in range(3):
        first = (i - 3 + k) if side == "-" else (i - 2 + k)
        cells = list(range(first, first + 3))
        coef = cell_average_poly([x_vals[j] for j in cells] + [x_vals[cells[-1] + 1]],
                                 [dplus[j] for j in cells])
        cands.append(float(peval(coef, x_vals[i])))
        if weights == "arclength":
            d1 = pderiv(coef)
            lo, hi = (i - 1, i) if side == "-" else (i, i + 1)
            uL, uR = float(peval(d1, x_vals[lo])), float(peval(d1, x_vals[hi]))
            L = arc_length_linear_slope(uL, uR, float(x_vals[hi] - x_vals[lo]))
            betas.append(L * L)
    if weights == "jp":
        if side == "-":
            v = [float(dplus[j]) for j in range(i - 3, i + 2)]
            betas = _jp_is(v)
        else:
            w = [float(dplus[j]) for j in range(i + 2, i - 3, -1)]
            betas = _jp_is(w)[::-1]   # mirrored index -> left-to-right index
    d = D_MINUS if side == "-" else D_PLUS
    al = [float(d[k]) / (eps + betas[k]) ** 2 for k in range(3)]
    om = [a / sum(al) for a in al]
    return sum(o * c for o, c in zip(om, cands)), cands, betas, om


def _jp_is(v):
    a, b, c, d = v[1] - v[0], v[2] - v[1], v[3] - v[2], v[4] - v[3]
    return [13 * (a - b) ** 2 + 3 * (a - 3 * b) ** 2,
            13 * (b - c) ** 2 + 3 * (b + c) ** 2,
            13 * (c - d) ** 2 + 3 * (3 * c - d) ** 2]


def extend(line, bc: str, g: int = 3):
    """Line of Fractions with g ghost values on each side (periodic or linear extrapolation)."""
    n = len(line)
    out = []
    for i in range(-g, n + g):
        if 0 <= i < n:
            out.append(line[i])
        elif bc == "periodic":
            out.append(line[i % n])
        elif i < 0:
            m = -i
            out.append((1 + m) * line[0] - m * line[1])
        else:
            m = i - (n - 1)
            out.append((1 + m) * line[n - 1] - m * line[n - 2])
    return out


def line_derivs(line, x0, dx, bc, weights, eps):
    """(phi_x^-, phi_x^+) at every node of a line (floats in, floats out)."""
    n = len(line)
    ext = extend([Fr(v) for v in line], bc)
    xs = [Fr(x0) + (j - 3) * Fr(dx) for j in range(n + 6)]
    um, up = np.zeros(n), np.zeros(n)
    for i in range(n):
        um[i] = one_sided(ext, xs, i + 3, "-", weights, eps)[0]
        up[i] = one_sided(ext, xs, i + 3, "+", weights, eps)[0]
    return um, up


def L_grid(phi, dx, dy, bc, weights, eps, Hfun, Hp, Hq, alpha: str, x0=0.37, y0=-0.61):
    """L = -Hhat (Lax-Friedrichs) on a whole 1D (shape (n,)) or 2D (ny, nx) grid.

    alpha: 'local' (per node, over the four (u, v) combinations) or 'global'
    (the grid maximum of the same values)."""
    phi = np.atleast_2d(np.asarray(phi, dtype=np.float64))
    ny, nx = phi.shape
    two_d = ny > 1
    um, up = np.zeros_like(phi), np.zeros_like(phi)
    vm, vp = np.zeros_like(phi), np.zeros_like(phi)
    for j in range(ny):
        um[j], up[j] = line_derivs(phi[j], x0, dx, bc, weights, eps)
    if two_d:
        for i in range(nx):
            vm[:, i], vp[:, i] = line_derivs(phi[:, i], y0, dy, bc, weights, eps)
    ax = np.zeros_like(phi)
    ay = np.zeros_like(phi)
    for u in (um, up):
        for v in (vm, vp):
            ax = np.maximum(ax, np.abs(Hp(u, v)))
            ay = np.maximum(ay, np.abs(Hq(u, v)))
    if not two_d:
        ay[:] = 0.0
    if alpha == "global":
        ax[:] = ax.max()
        ay[:] = ay.max()
    Hhat = Hfun(0.5 * (up + um), 0.5 * (vp + vm)) - ax * 0.5 * (up - um) - ay * 0.5 * (vp - vm)
    out = -Hhat
    return out if two_d else out[0]
