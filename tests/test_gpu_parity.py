"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

FP64: max-norm relative error <= 1e-12.  FP32 and MIXED: the bounds derived
for float stencil arithmetic, stated per test (one stage: a few float
rounding units of phi, amplified by the dt * dH/dp * d(phi_x)/d(phi) factor
of the stencil, which is O(1) under the CFL condition).
"""
import math

import numpy as np
import pytest

import oracle
from gpucase import Case, oracle_stages, rel_err
from paper_1909_13263_gb300 import inputs, native

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
# one RK stage in float arithmetic: |delta phi| <= dt |H_p| |delta phi_x| + rounding(phi)
# with |delta phi_x| ~ 8 u |phi| / dx (u = 2^-24) and dt |H_p| <= cfl dx: about 5 u |phi|,
# plus indicator perturbations near kinks; bound taken as 64 u = 3.8e-6
F32_STAGE_TOL = 64 * 2.0**-24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()
    native.use_torch_allocator(True)
    yield


CASES_2D = [
    Case(2, 70, 37, "burgers2d"),
    Case(2, 70, 37, "negcos2d", bc="linextrap"),
    Case(2, 45, 66, "sin2d", bc="linextrap", alpha_mode="local_lagged"),
    Case(2, 33, 17, "eikonal2d", alpha_mode="global_exact"),
    Case(2, 40, 40, "burgers2d", alpha_mode="fixed", alpha_fixed=(3.0, 2.5)),
    Case(2, 7, 5, "negcos2d"),
    Case(2, 3, 9, "burgers2d"),
    Case(2, 45, 38, "optctrl2d", lo=-math.pi, hi=math.pi),
    Case(2, 40, 33, "optctrl2d", lo=-math.pi, hi=math.pi, alpha_mode="local_lagged"),
]
CASES_1D = [
    Case(1, 300, 1, "burgers1d", alpha_mode="local_lagged"),
    Case(1, 20, 1, "negcos1d", alpha_mode="local_lagged"),
    Case(1, 257, 1, "advect1d", bc="linextrap", alpha_mode="global_lagged"),
    Case(1, 5, 1, "burgers1d", alpha_mode="global_exact"),
    Case(1, 130, 1, "nonconvex1d", alpha_mode="local_lagged"),
]


def _ids(c):
    return f"{c.dim}d-{c.nx}x{c.ny}-{c.ham}-{c.bc}-{c.alpha_mode}"


def _stage_dt(case, phi0):
    a, _ = oracle.alpha_of(case.cfg(), phi0)
    den = a[0] / case.dx + (a[1] / case.dy if case.dim == 2 else 0.0)
    return 0.6 / den


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("case", CASES_2D + CASES_1D, ids=_ids)
def test_fp64_rk_stages_match_oracle(case, weights):
    case.weights = weights
    phi0 = case.field(seed=3)
    dt = _stage_dt(case, phi0)
    ref = oracle_stages(case, phi0, dt)
    with case.solver() as s:
        s.set_phi0(phi0)
        s.run_stage(1, dt)
        e1 = rel_err(s.get_stage_phi(1), ref[0])
        s.run_stage(2, dt)
        e2 = rel_err(s.get_stage_phi(2), ref[1])
        s.run_stage(3, dt)
        e3 = rel_err(s.get_phi(), ref[2])
    assert max(e1, e2, e3) <= FP64_TOL, (e1, e2, e3)


@pytest.mark.parametrize("case", [
    Case(2, 70, 37, "burgers2d", weights="arclength"),
    Case(2, 70, 37, "negcos2d", weights="jp", bc="linextrap"),
    Case(2, 64, 40, "sin2d", alpha_mode="local_lagged", bc="linextrap"),
    Case(2, 40, 40, "burgers2d", alpha_mode="global_exact", dt_mode="dx53"),
    Case(2, 40, 32, "negcos2d", alpha_mode="local_exact"),
    Case(1, 80, 1, "burgers1d", alpha_mode="local_lagged"),
    Case(1, 300, 1, "negcos1d", alpha_mode="local_exact", dt_mode="dx53"),
], ids=_ids)
def test_fp64_solve_matches_oracle(case):
    # several whole steps, the last clipped to t_final, with the device-side dt rule
    phi0 = case.field(seed=5, kind="smooth")
    tf = 12 * _stage_dt(case, phi0) + 1e-4
    ref, steps_ref, t_ref, _, st = oracle.solve(case.cfg(), phi0, tf)
    assert st == 0
    with case.solver() as s:
        s.set_phi0(phi0)
        steps = s.step_to(tf)
        phi = s.get_phi()
        state = s.get_state()
    assert steps == steps_ref
    assert state.t == t_ref == tf
    assert rel_err(phi, ref) <= FP64_TOL


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("case", [
    Case(2, 150, 70, "burgers2d"),
    Case(2, 150, 70, "negcos2d", bc="linextrap"),
    Case(2, 65, 33, "sin2d", alpha_mode="local_lagged"),
    Case(1, 300, 1, "burgers1d", alpha_mode="local_lagged"),
    Case(1, 257, 1, "advect1d", bc="linextrap", alpha_mode="global_lagged"),
    Case(2, 130, 70, "optctrl2d", lo=-math.pi, hi=math.pi),
    Case(2, 70, 66, "optctrl2d", lo=-math.pi, hi=math.pi, alpha_mode="local_lagged"),
    Case(2, 97, 45, "eikonal2d", lo=0.0, hi=1.0),
    Case(2, 70, 66, "eikonal2d", bc="linextrap", alpha_mode="local_lagged"),
], ids=_ids)
def test_float_rk_stages_within_bound(case, weights, precision):
    case.weights, case.precision = weights, precision
    phi0 = case.field(seed=4)
    dt = _stage_dt(case, phi0)
    ref = oracle_stages(case, phi0, dt)
    with case.solver() as s:
        s.set_phi0(phi0)
        errs = []
        for stage in (1, 2, 3):
            s.run_stage(stage, dt)
            got = s.get_stage_phi(stage) if stage < 3 else s.get_phi()
            errs.append(rel_err(got, ref[stage - 1]))
    assert max(errs) <= F32_STAGE_TOL, errs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("kind", ["constant", "linear"])
def test_degenerate_data_stages_match_oracle(kind, weights, precision):
    # constant data (every difference zero: the vanishing-interval branch of the arc-length means and
    # zero Jiang-Peng indicators) and linear data (every second difference zero), where each stage
    # is phi + dt L with L = -H(a, b) at every node
    nx, ny = 70, 37
    if kind == "constant":
        case = Case(2, nx, ny, "negcos2d", weights=weights, precision=precision)
        phi0 = np.full((ny, nx), 0.7)
    else:
        case = Case(2, nx, ny, "burgers2d", bc="linextrap", weights=weights, precision=precision)
        x, _ = inputs.axis(nx, -1.0, 1.0, "linextrap")
        y, _ = inputs.axis(ny, -1.0, 1.0, "linextrap")
        X, Y = np.meshgrid(x, y, indexing="xy")
        phi0 = 0.3 * X - 0.45 * Y + 0.2
    dt = _stage_dt(case, phi0)
    ref = oracle_stages(case, phi0, dt)
    tol = FP64_TOL if precision == "fp64" else F32_STAGE_TOL
    with case.solver() as s:
        s.set_phi0(phi0)
        errs = []
        for stage in (1, 2, 3):
            s.run_stage(stage, dt)
            got = s.get_stage_phi(stage) if stage < 3 else s.get_phi()
            errs.append(rel_err(got, ref[stage - 1]))
    assert max(errs) <= tol, errs


def test_mixed_keeps_double_class_phi_between_steps():
    # phi^n round-trips through the (hi, lo) pair with about 48 significant bits
    case = Case(2, 70, 37, "burgers2d", precision="mixed")
    phi0 = case.field(seed=9, kind="smooth") + 1000.0
    with case.solver() as s:
        s.set_phi0(phi0)
        back = s.get_phi()
    assert rel_err(back, phi0) <= 2.0**-47


def test_mixed_solve_error_vs_fp64_oracle_is_bounded():
    # Example 3 on 160^2 to t = 0.5/pi^2: mixed error against the FP64 oracle stays
    # far below the discretisation error, and FP32 accumulation is visibly worse
    case = Case(2, 160, 160, "burgers2d", lo=-2.0, hi=2.0)
    x, dx = inputs.axis(160, -2.0, 2.0, "periodic")
    phi0 = inputs.phi0_negcos_diag_2d(x, x)
    tf = 0.5 / math.pi**2
    ref, steps_ref, _, _, st = oracle.solve(case.cfg(), phi0, tf)
    errs = {}
    for prec in ("mixed", "fp32"):
        case.precision = prec
        with case.solver() as s:
            s.set_phi0(phi0)
            s.step_to(tf)
            errs[prec] = float(np.max(np.abs(s.get_phi() - ref)))
    assert errs["mixed"] < 2e-6, errs
    assert errs["mixed"] <= errs["fp32"], errs
