"""The CUDA path on Examples 5, 8 and 11 of Sec. 3 at the paper's sizes, FP64,
against the oracle element by element (and against exact solutions where known).

Example 5: linear advection of a profile with corners, N = 100, to t = 2 and t = 8.
Example 8: the non-convex H = (p^2-1)(p^2-4)/4 from phi0 = -2|x| to t = 1, N = 100,
where the node alpha is the maximum of |H_p| over the interval between u^- and u^+.
Example 11: the optimal-control H(x, y, p, q) on [-pi, pi)^2 from phi0 = 0 to t = 1, 60^2.
"""
import math

import numpy as np
import pytest

import oracle
from gpucase import Case, rel_err
from paper_1909_13263_gb300 import inputs, native

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()
    native.use_torch_allocator(True)
    yield


def _solve_both(case, phi0, tf):
    ref, steps, t, _, st = oracle.solve(case.cfg(), phi0, tf)
    assert st == 0 and t == tf
    with case.solver() as s:
        s.set_phi0(phi0)
        assert s.step_to(tf) == steps
        got = s.get_phi()
        assert s.get_state().t == tf
    return got, ref


@pytest.mark.parametrize("t_final", [2.0, 8.0])
def test_example5_corners_match_oracle_and_resolve_corners(t_final):
    n = 100
    x, _ = inputs.axis(n, -1.0, 1.0, "periodic")
    phi0 = inputs.phi0_corners_1d(x)
    ex = inputs.phi0_corners_1d(x - t_final)
    err = {}
    for w in ("arclength", "jp"):
        case = Case(1, n, 1, "advect1d", weights=w, alpha_mode="default")
        got, ref = _solve_both(case, phi0, t_final)
        assert rel_err(got, ref) <= FP64_TOL, w
        err[w] = np.abs(got - ex)
    for c in (0.5 - 1.0 / 3.0, 0.5 + 1.0 / 3.0, -0.5):
        near = np.abs(((x - c + 1.0) % 2.0) - 1.0) < 0.1
        assert err["arclength"][near].max() < err["jp"][near].max()


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_example8_nonconvex_matches_oracle(weights):
    n = 100
    x, _ = inputs.axis(n, -1.0, 1.0, "periodic")
    case = Case(1, n, 1, "nonconvex1d", weights=weights, alpha_mode="default")
    got, ref = _solve_both(case, inputs.phi0_abs_1d(x), 1.0)
    assert rel_err(got, ref) <= FP64_TOL
    # the flattened top: phi(0, t) is near -t H(0) = -1 and the profile stays below it
    assert abs(got[n // 2] + 1.0) < 0.05 and got.max() < -0.9


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_example8_interval_alpha_stage_parity(precision):
    # slopes spread around sqrt(5/6) so that at many nodes the interior extremum of H_p,
    # not an end point, sets the node alpha
    n = 257
    x, _ = inputs.axis(n, -1.0, 1.0, "linextrap")
    rng = np.random.default_rng(85)
    phi0 = 0.913 * x + 0.004 * np.cumsum(rng.standard_normal(n))
    case = Case(1, n, 1, "nonconvex1d", bc="linextrap", alpha_mode="local_lagged", precision=precision)
    cfg = case.cfg()
    um, up, _, _ = oracle.derivs(cfg, phi0)
    c = np.sqrt(5.0 / 6.0)
    straddle = (np.minimum(um, up) < c) & (np.maximum(um, up) > c)
    hp = lambda p: np.abs(p**3 - 2.5 * p)
    interior_wins = straddle & (np.maximum(hp(um), hp(up)) < hp(c) - 1e-3)
    assert interior_wins.sum() >= 10
    a, _ = oracle.alpha_of(cfg, phi0)
    dt = 0.6 * case.dx / a[0]
    ref1 = phi0 + dt * oracle.L_of(cfg, phi0, a)
    with case.solver() as s:
        s.set_phi0(phi0)
        s.run_stage(1, dt)
        got1 = s.get_stage_phi(1)
    tol = FP64_TOL if precision == "fp64" else 64 * 2.0**-24
    assert rel_err(got1, ref1) <= tol


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_example11_optimal_control_matches_oracle(weights):
    n = 60
    case = Case(2, n, n, "optctrl2d", weights=weights, lo=-math.pi, hi=math.pi, alpha_mode="default")
    got, ref = _solve_both(case, np.zeros((n, n)), 1.0)
    assert rel_err(got, ref) <= FP64_TOL
    # the running cost is non-negative and phi0 = 0, so phi grows from 0 where the cost is positive
    assert got.min() > -0.05 and got.max() > 0.5


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_example11_float_paths_track_fp64(precision):
    # the position-dependent H in the float tile kernel (coordinates formed per node in float)
    n = 96
    out = {}
    for prec in ("fp64", precision):
        case = Case(2, n, n, "optctrl2d", lo=-math.pi, hi=math.pi, alpha_mode="default", precision=prec)
        with case.solver() as s:
            s.set_phi0(np.zeros((n, n)))
            s.step_to(0.5)
            out[prec] = s.get_phi()
    assert np.max(np.abs(out[precision] - out["fp64"])) < 1e-4


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("name", ["ex10_sin2d", "ex12_eikonal2d"])
def test_examples_10_12_at_paper_size_match_oracle(name, weights):
    # Example 10 (sin(p+q), pi(|y|-|x|), linear extrapolation, t = 1) and Example 12 (Eikonal,
    # [0, 1)^2 periodic, t = 0.6) on the paper's 80^2 grids, FP64, whole solves
    pr = inputs.PROBLEMS[name]
    n = 80
    phi0, _ = inputs.initial(pr, n)
    case = Case(2, n, n, pr.ham, bc=pr.bc, weights=weights, lo=pr.lo, hi=pr.hi, alpha_mode="default")
    got, ref = _solve_both(case, phi0, pr.t_final)
    assert rel_err(got, ref) <= FP64_TOL
