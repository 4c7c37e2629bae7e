"""The whole oracle scheme against the paper's accuracy tables and exact solutions.

Tables 1-4 (Sec. 3, Examples 1-4) print L-infinity and L1 errors; the oracle
reproduces them within a stated factor under the readings of the time step
(dt = 0.6 dx^{5/3} / alpha for convergence studies), of alpha (local in 1D,
grid-wide in 2D) and of the L1 norm (dx * sum in 1D, mean in 2D).
"""
import math
import os

import numpy as np
import pytest

import exact
import oracle
from paper_1909_13263_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TF = 0.5 / math.pi**2


def _table(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[int(v[0])] = {"arclength": (float(v[1]), float(v[2])), "jp": (float(v[3]), float(v[4]))}
    return rows


def _run_1d(ham, n, weights, t_final, exact_fn, alpha_mode="local_lagged"):
    x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
    cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham=ham, weights=weights, dt_mode="dx53", alpha_mode=alpha_mode)
    phi, steps, t, _, st = oracle.solve(cfg, inputs.phi0_negcos_1d(x), t_final)
    assert st == 0 and t == t_final
    e = np.abs(phi - exact_fn(x))
    return e.max(), dx * e.sum()


def _run_2d(ham, n, weights, alpha_mode="global_lagged"):
    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    cfg = oracle.make_cfg(dim=2, nx=n, ny=n, dx=dx, ham=ham, weights=weights, dt_mode="dx53",
                          alpha_mode=alpha_mode)
    phi, steps, t, _, st = oracle.solve(cfg, inputs.phi0_negcos_diag_2d(x, x), TF)
    assert st == 0 and t == TF
    e = np.abs(phi - exact.negcos_diag_2d(ham, x, x, TF))
    return e.max(), e.mean()


def _check(errs, table, weights, factor, factor_l1=None):
    factor_l1 = factor if factor_l1 is None else factor_l1
    for n, (linf, l1) in errs.items():
        p_linf, p_l1 = table[n][weights]
        assert p_linf / factor < linf < p_linf * factor, (n, linf, p_linf)
        assert p_l1 / factor_l1 < l1 < p_l1 * factor_l1, (n, l1, p_l1)


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_table1_linear_advection(weights):
    tab = _table("table1_ex1_advection.txt")
    errs = {n: _run_1d("advect1d", n, weights, 2.0, lambda x: -np.cos(np.pi * (x - 2.0)))
            for n in (20, 40, 80, 160)}
    _check(errs, tab, weights, 1.6)
    orders = [math.log2(errs[n][0] / errs[2 * n][0]) for n in (40, 80)]
    assert min(orders) > 4.8


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_table2_negcos_1d(weights):
    tab = _table("table2_ex2_negcos1d.txt")
    errs = {n: _run_1d("negcos1d", n, weights, TF, lambda x: exact.negcos_1d("negcos1d", x, TF))
            for n in (20, 40, 80, 160, 320)}
    _check(errs, tab, weights, 1.3)


def test_table2_needs_local_alpha():
    # the grid-wide alpha is 2-5x too dissipative for Table 2: pins the local reading in 1D
    tab = _table("table2_ex2_negcos1d.txt")
    linf, _ = _run_1d("negcos1d", 80, "arclength", TF, lambda x: exact.negcos_1d("negcos1d", x, TF),
                      alpha_mode="global_lagged")
    assert linf > 2.5 * tab[80]["arclength"][0]


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("ham,table", [("burgers2d", "table3_ex3_burgers2d.txt"),
                                       ("negcos2d", "table4_ex4_negcos2d.txt")])
def test_tables3_4_two_dimensional(ham, table, weights):
    tab = _table(table)
    errs = {n: _run_2d(ham, n, weights) for n in (20, 40, 80)}
    # the 2D L1 normalisation is not stated: the mean of |e| is within 2.5x, dx*dy*sum is not
    _check(errs, tab, weights, 2.0, 2.5)


def test_burgers_1d_smooth_fifth_order():
    # Example 6 before the kink forms: order close to 5 against characteristics
    ex = lambda x: exact.negcos_1d("burgers1d", x, TF)
    e = [_run_1d("burgers1d", n, "arclength", TF, ex)[0] for n in (80, 160, 320)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[-1] > 4.5, orders


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_burgers_1d_kink_is_non_oscillatory(weights):
    # Example 6 at t = 3.5/pi^2: a kink has formed; the solution stays bounded by the
    # Hopf-Lax bounds (no new extrema above max phi0 or below min phi0 - t max H)
    n = 80
    x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
    cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham="burgers1d", weights=weights, alpha_mode="local_lagged")
    tk = 3.5 / math.pi**2
    phi, _, t, _, st = oracle.solve(cfg, inputs.phi0_negcos_1d(x), tk)
    assert st == 0 and np.all(np.isfinite(phi))
    # phi_t = -(phi_x+1)^2/2 <= 0: phi never increases; and the kink stays a corner
    assert phi.max() <= 1.0 + 1e-12
    d2 = np.diff(phi, 2)
    assert np.sum(np.abs(np.diff(np.sign(d2[np.abs(d2) > 1e-3]))) > 0) <= 6


def test_example5_initial_data_is_continuous_and_periodic():
    # the third piece read as 15/2 - 3cos(2 pi x): continuous at the corners, periodic on [-1, 1)
    f = inputs.phi0_corners_1d
    for c in (0.5 - 1.0 / 3.0, 0.5, 0.5 + 1.0 / 3.0, -0.5):
        assert abs(f(c - 1e-12) - f(c)) < 1e-9
    assert abs(f(-1.0) - f(1.0 - 1e-13)) < 1e-9
    # corners: one-sided slopes differ at x - 0.5 = -1/3 and 1/3, agree at 0
    h = 1e-7
    slope = lambda c: ((f(c + h) - f(c)) / h, (f(c) - f(c - h)) / h)
    for c, corner in ((0.5 - 1.0 / 3.0, True), (0.5, False), (0.5 + 1.0 / 3.0, True)):
        r, l = slope(c)
        assert (abs(r - l) > 1.0) == corner


@pytest.mark.parametrize("t_final", [2.0, 8.0])
def test_example5_arclength_sharper_at_corners(t_final):
    # Example 5 (N = 100, CFL 0.6): the exact solution is phi0(x - t); near each corner of
    # the profile the arc-length weights give a smaller error than the Jiang-Peng weights
    n = 100
    x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
    ex = inputs.phi0_corners_1d(x - t_final)
    err = {}
    for w in ("arclength", "jp"):
        cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham="advect1d", weights=w, alpha_mode="local_lagged")
        phi, _, t, _, st = oracle.solve(cfg, inputs.phi0_corners_1d(x), t_final)
        assert st == 0 and t == t_final
        err[w] = np.abs(phi - ex)
    for c in (0.5 - 1.0 / 3.0, 0.5 + 1.0 / 3.0, -0.5):
        near = np.abs(((x - c + 1.0) % 2.0) - 1.0) < 0.1
        assert err["arclength"][near].max() < err["jp"][near].max()
    assert err["arclength"].max() < 1.0


def _hopf_example8(x, t):
    # phi0 = -2|x| is concave: psi = -phi has convex data 2|x| whose conjugate is 0 on [-2, 2],
    # so Hopf's formula gives phi(x, t) = -max_{|q| <= 2} (x q + t H(q)) on the whole line
    q = np.linspace(-2.0, 2.0, 200001)
    hq = 0.25 * (q * q - 1.0) * (q * q - 4.0)
    return np.array([-np.max(xi * q + t * hq) for xi in x])


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_example8_nonconvex_matches_hopf_formula(weights):
    # Example 8 on the periodic grid up to t = 0.15: with |H_p| <= 3 on [-2, 2] the corners of
    # the periodic profile at x = +-1 do not reach |x| <= 0.4, where Hopf's formula holds
    tf = 0.15
    l1 = []
    for n in (100, 200, 400):
        x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
        cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham="nonconvex1d", weights=weights, alpha_mode="local_lagged")
        phi, _, t, _, st = oracle.solve(cfg, inputs.phi0_abs_1d(x), tf)
        assert st == 0 and t == tf
        near = np.abs(x) <= 0.4
        e = np.abs(phi - _hopf_example8(x, tf))[near]
        l1.append(dx * e.sum())
        if n == 400:
            assert e.max() < 5e-3
    assert l1[0] / l1[1] > 1.7 and l1[1] / l1[2] > 1.7, l1


def _taylor_example11(X, Y, t):
    # phi0 = 0 and phi_t = -H(x, y, grad phi): phi = t l - t^2/2 (sin y l_x + sin x l_y + |l_y|) + O(t^3)
    # with l = sin^2(y)/2 + 1 - cos x the running cost (H(x, y, 0) = -l)
    lx, ly = np.sin(X), np.sin(Y) * np.cos(Y)
    ell = 0.5 * np.sin(Y) ** 2 + 1.0 - np.cos(X)
    return t * ell - 0.5 * t * t * (np.sin(Y) * lx + np.sin(X) * ly + np.abs(ly))


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_example11_short_time_expansion(weights):
    # Example 11 on [-pi, pi)^2 from phi0 = 0: the oracle matches the two-term expansion in t
    # with an O(t^3) remainder (ratio ~ 8 per halving of t), which fails if any term of H,
    # its position dependence or the sign convention of (sign q) q is wrong
    n = 40
    x, dx = inputs.axis(n, -np.pi, np.pi, "periodic")
    X, Y = np.meshgrid(x, x, indexing="xy")
    errs = []
    for tau in (0.1, 0.05):
        cfg = oracle.make_cfg(dim=2, nx=n, ny=n, dx=dx, dy=dx, ham="optctrl2d", weights=weights,
                              alpha_mode="global_lagged", xlo=-np.pi, ylo=-np.pi)
        phi, _, t, _, st = oracle.solve(cfg, np.zeros((n, n)), tau)
        assert st == 0 and t == tau
        e = np.abs(phi - _taylor_example11(X, Y, tau)).max()
        assert e < 1.5 * tau**3, (tau, e)
        errs.append(e)
    assert errs[0] / errs[1] > 6.0, errs


def _hopf_lax_example12(x, y, t):
    # H = sqrt(1 + |p|^2) is convex with Legendre transform L(v) = -sqrt(1 - |v|^2) on the unit disk, so
    # phi(x, t) = min over |v| <= 1 of phi0(x - t v) + t L(v): a polar grid, then a local refinement
    from scipy.optimize import minimize

    def phi0(a, b):
        return 0.25 * (np.cos(2 * np.pi * a) - 1.0) * (np.cos(2 * np.pi * b) - 1.0) - 1.0

    r = np.linspace(0.0, 1.0, 121)[:, None]
    a = np.linspace(0.0, 2.0 * np.pi, 241)[None, :]
    vx, vy = (r * np.cos(a)).ravel(), (r * np.sin(a)).ravel()
    f = phi0(x - t * vx, y - t * vy) - t * np.sqrt(np.maximum(0.0, 1.0 - vx * vx - vy * vy))
    k = int(np.argmin(f))

    def g(v):
        rr = v[0] * v[0] + v[1] * v[1]
        return phi0(x - t * v[0], y - t * v[1]) - t * np.sqrt(max(0.0, 1.0 - rr)) + 1e3 * max(0.0, rr - 1.0)

    res = minimize(g, [vx[k], vy[k]], method="Nelder-Mead", options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 4000})
    return min(res.fun, f[k])


def test_example12_eikonal_matches_hopf_lax():
    # Example 12 on [0, 1)^2 at t = 0.1 (arc-length weights, grid-wide alpha) against the Hopf-Lax formula at
    # 64 sample nodes: the mean error halves with the grid (a kink forms where phi0 has its maximum)
    t = 0.1
    means = []
    for n in (40, 80, 160):
        x, dx = inputs.axis(n, 0.0, 1.0, "periodic")
        cfg = oracle.make_cfg(dim=2, nx=n, ny=n, dx=dx, dy=dx, ham="eikonal2d", alpha_mode="global_lagged")
        phi, _, tt, _, st = oracle.solve(cfg, inputs.phi0_eikonal_2d(x, x), t)
        assert st == 0 and tt == t
        idx = [(i, j) for i in range(0, n, n // 8) for j in range(0, n, n // 8)]
        errs = [abs(phi[j, i] - _hopf_lax_example12(x[i], x[j], t)) for i, j in idx]
        means.append(float(np.mean(errs)))
        assert max(errs) < 0.02
    assert means[1] < 1.5e-4 and means[0] / means[1] > 1.5 and means[1] / means[2] > 1.5, means
