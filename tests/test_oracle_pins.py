"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: exact
rational solves of the paper's cell-average conditions (Steps 1-2), the
printed coefficient tables, quadrature of the arc-length integral (Eq. length),
polynomial exactness, the weight-accuracy claim of Step 4, consistency of the
Lax-Friedrichs Hamiltonian, the RK3 amplification polynomial (Step 5), and an
independent brute-force restatement on tiny grids.
"""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import bruteforce as bf
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "coefficients.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, vals = line.split(":")
        out[key.strip()] = [Fr(v) for v in vals.split()]
    return out


def _coeffs_of(cells, xi):
    """Coefficients on Delta^+ phi_j (j in cells) of p(x_i), p solving the cell averages."""
    xs = [Fr(j) for j in range(cells[0], cells[-1] + 2)]
    out = []
    for m in range(len(cells)):
        e = [Fr(int(r == m)) for r in range(len(cells))]
        out.append(bf.peval(bf.cell_average_poly(xs, e), Fr(xi)))
    return out


def test_step2_candidates_from_cell_averages():
    g = _golden()
    # S_k^- cells j = i-3+k .. i-1+k with i = 0; coefficients on Delta^+ phi_{i-3..i+1}
    for k in range(3):
        c = _coeffs_of(list(range(-3 + k, k)), 0)
        row = [Fr(0)] * 5
        row[k:k + 3] = c
        assert row == g[f"cand {k}"]


def test_step1_linear_combination_and_signs():
    g = _golden()
    big_minus = _coeffs_of(list(range(-3, 2)), 0)         # degree-4, cells i-3..i+1
    assert big_minus == g["step1 minus"]
    assert sum(big_minus) == 1
    combo = [sum(g["d"][k] * g[f"cand {k}"][m] for k in range(3)) for m in range(5)]
    assert combo == g["step1 minus"]
    big_plus = _coeffs_of(list(range(-2, 3)), 0)          # cells i-2..i+2
    assert big_plus == g["step1 plus"]
    # + side: left-to-right sub-stencils T_k^+ with the mirrored weights (3/10, 6/10, 1/10)
    plus_c = [_coeffs_of(list(range(-2 + k, 1 + k)), 0) for k in range(3)]
    combo_p = [Fr(0)] * 5
    for k, d in enumerate(bf.D_PLUS):
        for m, c in enumerate(plus_c[k]):
            combo_p[k + m] += d * c
    assert combo_p == g["step1 plus"]


def test_oracle_candidates_match_printed_coefficients():
    g = _golden()
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = rng.normal(size=6)
        dx = 10 ** rng.uniform(-3, -1)
        _, cand, _, _ = oracle.phix_minus(p, dx)
        v = np.diff(p) / dx
        for k in range(3):
            ref = sum(float(c) * vv for c, vv in zip(g[f"cand {k}"], v))
            assert cand[k] == pytest.approx(ref, rel=1e-13, abs=1e-13 * np.abs(v).max())


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("side", ["-", "+"])
def test_one_sided_matches_bruteforce(weights, side):
    rng = np.random.default_rng(7)
    dx = 0.05
    for trial in range(6):
        kind = trial % 3
        x0 = 0.73 + trial
        xs = [Fr(x0) + j * Fr(dx) for j in range(-3, 4)]   # x_{i-3..i+3}, i at index 3
        if kind == 0:
            vals = rng.normal(size=7)
        elif kind == 1:
            vals = np.sin(3.0 * np.array([float(x) for x in xs]))
        else:
            vals = np.abs(np.array([float(x) for x in xs]) - x0 - 0.01)
        ref = bf.one_sided([Fr(v) for v in vals], xs, 3, side, weights, 1e-6)
        if side == "-":
            got = oracle.phix_minus(vals[0:6], dx, weights)
        else:
            got = oracle.phix_plus(vals[1:7], dx, weights)
        # candidates and betas in the paper's left-to-right order for "+"
        cand = got[1] if side == "-" else got[1][::-1]
        beta = got[2] if side == "-" else got[2][::-1]
        omega = got[3] if side == "-" else got[3][::-1]
        np.testing.assert_allclose(cand, ref[1], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(beta, ref[2], rtol=1e-11, atol=1e-300)
        np.testing.assert_allclose(omega, ref[3], rtol=1e-11, atol=1e-15)
        assert got[0] == pytest.approx(ref[0], rel=1e-12, abs=1e-12)


def _gl_arclength(b, c, z0, z1):
    return bf.arc_length_linear_slope(b + 2 * c * z0, b + 2 * c * z1, z1 - z0)


def test_arclength_primitive_vs_quadrature():
    rng = np.random.default_rng(3)
    cases = [(1.0, 0.0, 0.0, 1.0), (0.3, 1e-12, -0.01, 0.0), (5.0, 2.0, -0.5, 0.0),
             (-40.0, 800.0, -0.02, 0.0), (0.0, 1e6, -1e-3, 0.0)]
    for _ in range(200):
        b = rng.normal() * 10 ** rng.uniform(-2, 3)
        c = rng.normal() * 10 ** rng.uniform(-8, 4)
        dz = 10 ** rng.uniform(-4, 0)
        cases.append((b, c, -dz, 0.0))
    for b, c, z0, z1 in cases:
        got = oracle.arclength(b, c, z0, z1)
        ref = _gl_arclength(b, c, z0, z1)
        assert got == pytest.approx(ref, rel=2e-13), (b, c, z0, z1)


def test_arclength_taylor_switch_is_continuous():
    # both sides of |u1-u0| = 1e-3 sqrt(1+m^2) agree with quadrature
    for m in (0.0, 0.7, -3.0, 50.0):
        s = math.sqrt(1 + m * m)
        for f in (0.999, 1.001):
            h = f * 1e-3 * s
            c = h / (2 * 0.01)
            b = m + h / 2
            got = oracle.arclength(b, c, -0.01, 0.0)
            assert got == pytest.approx(_gl_arclength(b, c, -0.01, 0.0), rel=1e-13)


def test_arclength_c_zero_branch():
    for b in (0.0, 1.0, -7.5):
        assert oracle.arclength(b, 0.0, -0.1, 0.0) == pytest.approx(0.1 * math.sqrt(1 + b * b), rel=1e-15)


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_polynomial_exactness_degree3(weights):
    rng = np.random.default_rng(11)
    dx, xi = 0.01, 0.42
    x = xi + dx * np.arange(-3, 4)
    for _ in range(10):
        a = rng.normal(size=4)
        phi = a[0] + a[1] * x + a[2] * x**2 + a[3] * x**3
        exact = a[1] + 2 * a[2] * xi + 3 * a[3] * xi**2
        scale = np.abs(phi).max() / dx
        vm = oracle.phix_minus(phi[0:6], dx, weights)[0]
        vp = oracle.phix_plus(phi[1:7], dx, weights)[0]
        assert abs(vm - exact) < 1e-12 * scale
        assert abs(vp - exact) < 1e-12 * scale


def test_linear_limit_is_fifth_order_exact():
    # eps >> beta drives omega to d: the Step-1 scheme, exact for degree <= 4 polynomials
    # (phi_x of degree <= 4 reconstructed from a degree-4 polynomial), one-sided both ways.
    rng = np.random.default_rng(12)
    dx, xi = 0.1, 0.3
    x = xi + dx * np.arange(-3, 4)
    for _ in range(10):
        a = rng.normal(size=6)
        phi = sum(a[m] * x**m for m in range(6))
        exact = sum(m * a[m] * xi ** (m - 1) for m in range(1, 6))
        for w in ("arclength", "jp"):
            vm = oracle.phix_minus(phi[0:6], dx, w, eps=1e12)[0]
            vp = oracle.phix_plus(phi[1:7], dx, w, eps=1e12)[0]
            assert vm == pytest.approx(exact, rel=1e-10, abs=1e-10)
            assert vp == pytest.approx(exact, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_weights_are_linear_on_cubics(weights):
    # on a cubic all three candidate polynomials p_i^k are the same quadratic, so the
    # arc-length indicators coincide (and so do the Jiang-Peng ones): omega = d exactly;
    # a quartic separates them
    dx = 0.05
    x = 0.2 + dx * np.arange(-3, 4)
    d = np.array([0.1, 0.6, 0.3])
    cubic = 0.3 - x + 2 * x**2 + 5 * x**3
    quartic = cubic + 40 * x**4
    for f, win in ((oracle.phix_minus, slice(0, 6)), (oracle.phix_plus, slice(1, 7))):
        np.testing.assert_allclose(f(cubic[win], dx, weights)[3], d, rtol=0, atol=1e-13)
        assert np.abs(f(quartic[win], dx, weights)[3] - d).max() > 1e-4


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_weights_converge_second_order(weights):
    # Step 4: omega_k = d_k + O(dx^2) on smooth data
    errs, dxs = [], [0.04, 0.02, 0.01, 0.005]
    for dx in dxs:
        x = 0.3 + dx * np.arange(-3, 3)
        phi = np.sin(2 * x) + 0.5 * np.exp(x)
        om = oracle.phix_minus(phi, dx, weights, eps=0.0)[3]
        errs.append(np.abs(om - np.array([0.1, 0.6, 0.3])).max())
    slopes = np.diff(np.log(errs)) / np.diff(np.log(dxs))
    assert np.all(np.abs(slopes - 2.0) < 0.25), slopes


def test_weights_convex_on_rough_data():
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = rng.normal(size=6) * 10 ** rng.uniform(-3, 3)
        for w in ("arclength", "jp"):
            om = oracle.phix_minus(p, 10 ** rng.uniform(-4, 0), w)[3]
            assert np.all(om >= 0) and np.all(om <= 1)
            assert om.sum() == pytest.approx(1.0, abs=1e-14)


HAMS2 = {
    "burgers2d": (lambda p, q, x, y: 0.5 * (p + q + 1) ** 2),
    "negcos2d": (lambda p, q, x, y: -np.cos(p + q + 1)),
    "sin2d": (lambda p, q, x, y: np.sin(p + q)),
    "eikonal2d": (lambda p, q, x, y: np.sqrt(p * p + q * q + 1)),
    "advect1d": (lambda p, q, x, y: p),
    "burgers1d": (lambda p, q, x, y: 0.5 * (p + 1) ** 2),
    "negcos1d": (lambda p, q, x, y: -np.cos(p + 1)),
    "nonconvex1d": (lambda p, q, x, y: 0.25 * (p * p - 1) * (p * p - 4)),
    # Example 11 with (sign q) q written as |q|
    "optctrl2d": (lambda p, q, x, y: np.sin(y) * p + np.sin(x) * q + abs(q) - 0.5 * np.sin(y) ** 2
                  - (1 - np.cos(x))),
}


@pytest.mark.parametrize("kind", list(HAMS2))
def test_hamiltonian_values_and_partials(kind):
    rng = np.random.default_rng(2)
    f = HAMS2[kind]
    for _ in range(20):
        p, q = rng.normal(size=2) * 2
        x, y = rng.uniform(-np.pi, np.pi, size=2)
        H, Hp, Hq = oracle.ham(kind, p, q, x, y)
        assert H == pytest.approx(f(p, q, x, y), rel=1e-14, abs=1e-14)
        h = 1e-6
        assert Hp == pytest.approx((f(p + h, q, x, y) - f(p - h, q, x, y)) / (2 * h), rel=1e-6, abs=1e-7)
        assert Hq == pytest.approx((f(p, q + h, x, y) - f(p, q - h, x, y)) / (2 * h), rel=1e-6, abs=1e-7)


@pytest.mark.parametrize("kind", list(HAMS2))
def test_lf_flux_consistent_and_monotone(kind):
    rng = np.random.default_rng(4)
    for _ in range(20):
        u, v = rng.normal(size=2)
        x, y = rng.uniform(-np.pi, np.pi, size=2)
        H = oracle.ham(kind, u, v, x, y)[0]
        assert oracle.hhat(kind, u, u, v, v, 3.0, 3.0, x, y) == pytest.approx(H, rel=1e-15, abs=1e-15)
        # non-increasing in u^+, non-decreasing in u^- when alpha bounds |H_p| on the range
        up, um, vp, vm = rng.normal(size=4) * 0.5
        a = 4.0  # bounds |H_p|, |H_q| of every kind on |p|, |q| <= 1.5
        h = 1e-6
        hh = lambda *d: oracle.hhat(kind, *d, a, a, x, y)
        d_up = hh(up + h, um, vp, vm) - hh(up, um, vp, vm)
        d_um = hh(up, um + h, vp, vm) - hh(up, um, vp, vm)
        d_vp = hh(up, um, vp + h, vm) - hh(up, um, vp, vm)
        d_vm = hh(up, um, vp, vm + h) - hh(up, um, vp, vm)
        assert d_up <= 1e-15 and d_um >= -1e-15 and d_vp <= 1e-15 and d_vm >= -1e-15


def test_optimal_control_alpha_bounds_the_slopes_of_H():
    # Example 11: alpha_x = |sin y|; alpha_y = the largest |dH/dq| over the interval between
    # v^- and v^+, where the kink of |q| at 0 contributes both one-sided slopes sin x +- 1
    f = HAMS2["optctrl2d"]
    rng = np.random.default_rng(11)
    for _ in range(300):
        x, y = rng.uniform(-np.pi, np.pi, size=2)
        um, up = rng.normal(size=2)
        vm, vp = rng.normal(size=2) * rng.choice([1e-3, 0.3, 2.0])
        if rng.random() < 0.1:
            vm = vp = 0.0
        ax, ay = oracle.node_alpha("optctrl2d", 2, um, up, vm, vp, x, y)
        assert ax == pytest.approx(abs(np.sin(y)), abs=1e-15)
        lo, hi = min(vm, vp), max(vm, vp)
        # one-sided difference quotients of H in q, sampled across [lo, hi]
        qs = np.linspace(lo, hi, 101)
        h = 1e-7
        slopes = [abs(f(0.1, qq + s * h, x, y) - f(0.1, qq, x, y)) / h for qq in qs for s in (1, -1)]
        assert ay == pytest.approx(max(slopes), rel=1e-5, abs=1e-6)
        # the flux built on it is monotone over the whole interval
        assert ay >= max(slopes) - 1e-6


def test_rk3_amplification_polynomial():
    # y' = A y with A a scaled rotation: one step multiplies by R(dt A), R(z) = 1+z+z^2/2+z^3/6
    for a, b, dt in ((-1.0, 0.0, 0.3), (-0.5, 2.0, 0.2), (0.0, 1.0, 0.9)):
        A = np.array([[a, -b], [b, a]])
        y0 = np.array([0.7, -0.2])
        got = oracle.rk3_step_generic(y0, dt, lambda y: A @ y)
        Z = dt * A
        R = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
        np.testing.assert_allclose(got, R @ y0, rtol=1e-14, atol=1e-15)


def _cfg1(n, dx, ham, weights, alpha_mode, bc="periodic"):
    return oracle.make_cfg(dim=1, nx=n, dx=dx, ham=ham, weights=weights, alpha_mode=alpha_mode, bc=bc)


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("alpha", ["local", "global"])
def test_tiny_1d_grid_L_matches_bruteforce(weights, alpha):
    rng = np.random.default_rng(21)
    n, dx = 8, 0.1
    phi = np.cos(2 * np.pi * np.arange(n) / n) + 0.3 * rng.normal(size=n)
    Hf = lambda p, q: 0.5 * (p + 1) ** 2
    ref = bf.L_grid(phi, dx, dx, "periodic", weights, 1e-6, Hf, lambda p, q: p + 1,
                    lambda p, q: 0 * p, alpha)
    cfg = _cfg1(n, dx, "burgers1d", weights, alpha + "_lagged")
    a, _ = oracle.alpha_of(cfg, phi)
    got = oracle.L_of(cfg, phi, a)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("bc", ["periodic", "linextrap"])
def test_tiny_2d_grid_L_matches_bruteforce(weights, bc):
    rng = np.random.default_rng(22)
    ny, nx, dx, dy = 7, 9, 0.125, 0.2
    phi = rng.normal(size=(ny, nx))
    Hf = lambda p, q: -np.cos(p + q + 1)
    Hp = lambda p, q: np.sin(p + q + 1)
    ref = bf.L_grid(phi, dx, dy, bc, weights, 1e-6, Hf, Hp, Hp, "global")
    cfg = oracle.make_cfg(dim=2, nx=nx, ny=ny, dx=dx, dy=dy, ham="negcos2d", weights=weights,
                          alpha_mode="global_lagged", bc=bc)
    a, _ = oracle.alpha_of(cfg, phi)
    got = oracle.L_of(cfg, phi, a)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_mirror_and_transpose_symmetry():
    rng = np.random.default_rng(31)
    n, dx = 24, 1.0 / 24
    phi = rng.normal(size=n)
    cfg = _cfg1(n, dx, "burgers1d", "arclength", "local_lagged")
    um, up, _, _ = oracle.derivs(cfg, phi)
    # psi_j = phi_{-j}: phi_x^+(phi)_i = -phi_x^-(psi)_{-i}
    idx = (-np.arange(n)) % n
    psi = phi[idx]
    pm, pp, _, _ = oracle.derivs(cfg, psi)
    np.testing.assert_allclose(up, -pm[idx], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(um, -pp[idx], rtol=1e-13, atol=1e-13)
    ph2 = rng.normal(size=(10, 13))
    c2 = oracle.make_cfg(dim=2, nx=13, ny=10, dx=0.1, dy=0.1, ham="burgers2d")
    ct = oracle.make_cfg(dim=2, nx=10, ny=13, dx=0.1, dy=0.1, ham="burgers2d")
    a = oracle.derivs(c2, ph2)
    b = oracle.derivs(ct, ph2.T.copy())
    np.testing.assert_array_equal(a[0], b[2].T)
    np.testing.assert_array_equal(a[1], b[3].T)


def test_nonconvex_alpha_is_the_interval_maximum():
    # Example 8's H_p = p^3 - 5p/2 is not monotone: alpha over [u^-, u^+] includes interior extrema
    rng = np.random.default_rng(8)
    for _ in range(200):
        um, up = rng.uniform(-2.5, 2.5, size=2)
        s = np.linspace(min(um, up), max(um, up), 20001)
        ref = np.max(np.abs(s**3 - 2.5 * s))
        got = oracle.node_alpha("nonconvex1d", 1, um, up)[0]
        assert got == pytest.approx(ref, rel=1e-6, abs=1e-9)
        assert got >= ref - 1e-12
    # for monotone-derivative Hamiltonians the node alpha is the end-point maximum
    for kind, hp in (("burgers1d", lambda p: abs(p + 1)), ("advect1d", lambda p: 1.0)):
        um, up = -0.7, 1.3
        assert oracle.node_alpha(kind, 1, um, up)[0] == pytest.approx(max(hp(um), hp(up)))


@pytest.mark.parametrize("dim,ham,bc,alpha", [(2, "burgers2d", "periodic", "global_lagged"),
                                              (2, "optctrl2d", "linextrap", "local_lagged"),
                                              (2, "sin2d", "linextrap", "fixed"),
                                              (1, "nonconvex1d", "periodic", "local_lagged")])
def test_single_node_L_matches_the_grid_L(dim, ham, bc, alpha):
    # the one-node operator (used to check sampled nodes of very large grids) is the grid operator
    # L = -H-hat of Eq. LF at that node, boundaries and node coordinates included
    rng = np.random.default_rng(11)
    nx, ny = (23, 17) if dim == 2 else (29, 1)
    phi = rng.standard_normal((ny, nx) if dim == 2 else nx)
    cfg = oracle.make_cfg(dim=dim, nx=nx, ny=ny, bc=bc, dx=0.13, dy=0.11, ham=ham, alpha_mode=alpha,
                          alpha_fixed=(1.0, 1.5), xlo=-1.3, ylo=0.4)
    a = np.array([1.7, 2.3])
    full = oracle.L_of(cfg, phi, a)
    for j in range(ny):
        for i in range(nx):
            one = oracle.point_L(cfg, phi, i, j, a)
            ref = full[j, i] if dim == 2 else full[i]
            assert one == pytest.approx(ref, rel=1e-14, abs=1e-14), (i, j)


def test_solve_rk3_translates_cubic_data_exactly():
    # Step 5 as orc_solve runs it: phi_t + phi_x = 0 (H = p, Example 1's equation) with cubic data on a
    # linear-extrapolation grid.  Every candidate of Step 2 is exact for cubics, so at nodes whose
    # stencils never reach a ghost, L = -phi_x exactly for any weights and the LF term vanishes
    # (u^+ = u^-).  One Shu-Osher step then gives phi - dt phi' + dt^2 phi''/2 - dt^3 phi'''/6,
    # the cubic translated by dt: each stage's dependence widens by three nodes, so nodes 9..n-10
    # must equal p(x - dt).  A wrong stage weight (3/4, 1/4, 1/3, 2/3) breaks this.
    rng = np.random.default_rng(1909)
    n, lo, hi = 41, -1.0, 1.0
    dx = (hi - lo) / (n - 1)
    x = lo + dx * np.arange(n)
    for _ in range(3):
        c = rng.normal(size=4)
        p = lambda z: c[0] + c[1] * z + c[2] * z**2 + c[3] * z**3
        cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham="advect1d", bc="linextrap", alpha_mode="fixed",
                              alpha_fixed=(1.0, 0.0), xlo=lo)
        dt = 0.37 * dx      # below the CFL step 0.6 dx: one (clipped) step
        phi, steps, t, _, st = oracle.solve(cfg, p(x), dt)
        assert st == 0 and steps == 1 and t == dt
        np.testing.assert_allclose(phi[9:n - 9], p(x[9:n - 9] - dt), rtol=0, atol=1e-13)
        # the boundary nodes use linearly extrapolated ghosts, which are not exact for cubics
        assert np.abs(phi[:3] - p(x[:3] - dt)).max() > 1e-9


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_linextrap_ghosts_exact_on_linear_data(weights):
    # The ghost values phi_{-m} = (1+m) phi_0 - m phi_1 (and the mirror image at the right end) extend
    # linear data exactly, so every one-sided derivative -- also at the three nodes next to each end,
    # whose stencils reach the ghosts -- equals the slope.  A wrong sign or index in a ghost fails here.
    rng = np.random.default_rng(7)
    n = 13
    dx = 0.25
    x = dx * np.arange(n)
    b = -0.4 - rng.random()    # slopes of order one: rounding of the data stays far below 1e-13
    cfg = oracle.make_cfg(dim=1, nx=n, dx=dx, ham="advect1d", bc="linextrap", weights=weights)
    um, up, _, _ = oracle.derivs(cfg, 0.3 + b * x)
    np.testing.assert_allclose(um, b, rtol=1e-13, atol=0)
    np.testing.assert_allclose(up, b, rtol=1e-13, atol=0)
    # 2D: slopes in both directions, ragged sizes
    ny, nx, dy = 9, 11, 0.2
    bx, by = 0.5 + rng.random(2)
    X, Y = np.meshgrid(dx * np.arange(nx), dy * np.arange(ny))
    cfg2 = oracle.make_cfg(dim=2, nx=nx, ny=ny, dx=dx, dy=dy, ham="burgers2d", bc="linextrap", weights=weights)
    um, up, vm, vp = oracle.derivs(cfg2, -1.1 + bx * X + by * Y)
    for a in (um, up):
        np.testing.assert_allclose(a, bx, rtol=1e-13, atol=0)
    for a in (vm, vp):
        np.testing.assert_allclose(a, by, rtol=1e-13, atol=0)
    # quadratic data is not extended exactly: the boundary derivatives differ from the exact ones
    q = 0.5 * x**2
    um, up, _, _ = oracle.derivs(cfg, q)
    assert abs(um[0] - 0.0) > 1e-3 and np.allclose(um[4:-4], x[4:-4], rtol=1e-12, atol=1e-12)
