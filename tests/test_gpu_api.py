"""C-ABI behaviour on the GPU: checkpoint/resume, error paths, full-size sampled
parity in the configuration bench.py times, and 1D / boundary workloads."""
import math
import os

import numpy as np
import pytest

import oracle
from gpucase import Case, rel_err
from paper_1909_13263_gb300 import inputs, native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()
    native.use_torch_allocator(True)
    yield


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_checkpoint_resume_reproduces_uninterrupted_run(precision):
    case = Case(2, 96, 80, "negcos2d", precision=precision, lo=-2.0, hi=2.0)
    phi0 = case.field(seed=12, kind="smooth")
    t1, t2 = 0.01, 0.025
    with case.solver() as a:
        a.set_phi0(phi0)
        a.step_to(t1)
        state = a.get_state()
        mid = a.get_phi()
        a.step_to(t2)
        full = a.get_phi()
        steps_full = a.get_state().steps
    with case.solver() as b:
        b.set_state(state, mid)
        b.step_to(t2)
        resumed = b.get_phi()
        assert b.get_state().steps == steps_full
    if precision == "mixed":
        # the (hi, lo) split of a checkpointed double is canonical up to a tie in rounding
        assert rel_err(resumed, full) <= 1e-14
    else:
        assert np.array_equal(resumed, full)


def test_results_into_caller_buffers_equal_returned_results():
    case = Case(2, 96, 80, "burgers2d", precision="mixed", lo=-2.0, hi=2.0)
    phi0 = case.field(seed=5, kind="smooth")
    with case.solver() as s:
        s.set_phi0(phi0)
        s.step_to(0.01)
        own = s.get_phi()
        buf = np.full(own.shape, np.nan)
        assert s.get_phi(out=buf) is buf
        assert np.array_equal(buf, own)
    kw = dict(xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0)
    with native.Batch(precision="mixed") as b:
        b.add(nx=96, ny=80, ham="burgers2d", phi0=phi0, t_final=0.01, **kw)
        b.add(nx=64, ny=64, ham="negcos2d", phi0=phi0[:64, :64].copy(), t_final=0.005, **kw)
        b.run()
        for k, shape in enumerate([(80, 96), (64, 64)]):
            buf = np.full(shape, np.nan)
            assert b.get_phi(k, out=buf) is buf
            assert np.array_equal(buf, b.get_phi(k))
        with pytest.raises(ValueError):
            b.get_phi(0, out=np.zeros((96, 80)))


def test_invalid_arguments_are_rejected():
    with pytest.raises(native.AlwError) as e:
        native.Solver(dim=2, nx=16, ny=16, xlo=0, xhi=1, ylo=0, yhi=1, ham="burgers1d")
    assert e.value.status == native.EINVAL
    with pytest.raises(native.AlwError) as e:
        native.Solver(dim=2, nx=1, ny=16, bc="linextrap", xlo=0, xhi=1, ylo=0, yhi=1, ham="burgers2d")
    assert e.value.status == native.EINVAL
    s = native.Solver(dim=2, nx=16, ny=16, xlo=0, xhi=1, ylo=0, yhi=1, ham="burgers2d")
    with pytest.raises(native.AlwError) as e:
        s.set_phi0(np.zeros(15 * 16))
    assert e.value.status == native.EINVAL
    with pytest.raises(native.AlwError) as e:
        s.step_to(1.0)  # phi0 not set
    assert e.value.status == native.EINVAL
    with pytest.raises(native.AlwError) as e:
        s.run_stage(4, 1e-3)
    assert e.value.status in (native.EINVAL,)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_finite_input_is_reported(precision):
    case = Case(2, 64, 64, "burgers2d", precision=precision)
    phi0 = case.field(seed=1, kind="smooth")
    phi0[10, 20] = np.nan
    with case.solver() as s:
        s.set_phi0(phi0)
        with pytest.raises(native.AlwError) as e:
            s.step_to(0.05)
        assert e.value.status == native.ENONFINITE


def test_no_progress_is_reported_as_timeout(monkeypatch):
    # host-side injection: the progress check of alw_step_to sees the device state frozen after its
    # first read (the device itself keeps working), so the call must give up with ALW_ETIMEOUT
    # instead of waiting; without the injection the same solver then finishes normally
    case = Case(2, 64, 48, "burgers2d", precision="mixed", lo=-2.0, hi=2.0)
    with case.solver() as s:
        s.set_phi0(case.field(seed=3, kind="smooth"))
        monkeypatch.setenv("ALW_TEST_FREEZE_STATE_AFTER", "1")
        with pytest.raises(native.AlwError) as e:
            s.step_to(0.2)
        assert e.value.status == native.ETIMEOUT
        monkeypatch.delenv("ALW_TEST_FREEZE_STATE_AFTER")
        s.step_to(0.2)
        assert s.get_state().t == 0.2


@pytest.mark.parametrize("precision,alpha", [("mixed", "fixed"), ("mixed", "local_lagged"), ("fp64", "fixed")])
def test_full_size_8192_sampled_stage_parity(precision, alpha):
    # the bench configuration (Example 3 on 8192^2): one RK stage on the GPU, checked at
    # sampled nodes (tile corners, grid edges, random interior) against the oracle's per-node L
    n = 8192
    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    case = Case(2, n, n, "burgers2d", lo=-2.0, hi=2.0, precision=precision, alpha_mode=alpha,
                alpha_fixed=(1.0 + math.pi, 1.0 + math.pi))
    phi0 = np.ascontiguousarray(inputs.phi0_negcos_diag_2d(x, x))
    dt = 0.6 / (2 * (1.0 + math.pi) / dx)
    with case.solver() as s:
        s.set_phi0(phi0)
        s.run_stage(1, dt)
        phi1 = s.get_stage_phi(1)
    rng = np.random.default_rng(8192)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (63, 31), (64, 32), (8191, 4095), (4096, 8191)]
    pts += [(int(i), int(j)) for i, j in rng.integers(0, n, size=(600, 2))]
    cfg = case.cfg()
    a = np.array(case.alpha_fixed)
    errs = []
    for i, j in pts:
        ref = phi0[j, i] + dt * oracle.point_L(cfg, phi0, i, j, a)
        errs.append(abs(phi1[j, i] - ref))
    err = max(errs) / np.abs(phi0).max()
    tol = 1e-12 if precision == "fp64" else 64 * 2.0**-24
    assert err <= tol, err


def test_large_ragged_linextrap_three_stages_sampled():
    # a large non-square grid with ragged tiles in both directions (12347 = 192 * 64 + 59 columns, 5003 =
    # 156 * 32 + 11 rows), dx != dy and linear-extrapolation ghosts (Example 10's Hamiltonian and data): every
    # stage of the MIXED path at sampled nodes -- the boundary bands, the ragged last tiles, tile seams and
    # random interior nodes -- against the oracle's per-node operator applied to the GPU's previous stage
    # state (stage 2 and 3 each checked on their own input)
    nx, ny = 12347, 5003
    case = Case(2, nx, ny, "sin2d", bc="linextrap", lo=-1.0, hi=1.0, precision="mixed", alpha_mode="fixed",
                alpha_fixed=(1.0, 1.0))
    x, dx = inputs.axis(nx, -1.0, 1.0, "linextrap")
    y, dy = inputs.axis(ny, -1.0, 1.0, "linextrap")
    phi0 = np.ascontiguousarray(inputs.phi0_riemann_2d(x, y))
    dt = 0.6 / (1.0 / dx + 1.0 / dy)
    with case.solver() as s:
        s.set_phi0(phi0)
        got = []
        for stage in (1, 2, 3):
            s.run_stage(stage, dt)
            got.append(s.get_stage_phi(stage) if stage < 3 else s.get_phi())
    rng = np.random.default_rng(12347)
    pts = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (1, 2), (2, 1), (nx - 2, ny - 3), (nx - 3, ny - 2),
           (63, 31), (64, 32), (12287, 4991), (12288, 4992), (nx // 2, ny // 2), (nx // 2 + 1, ny // 2 - 1)]
    pts += [(int(i), int(j)) for i, j in zip(rng.integers(0, nx, 300), rng.integers(0, ny, 300))]
    pts += [(int(i), int(j)) for i, j in zip(rng.integers(0, 3, 60), rng.integers(0, ny, 60))]
    pts += [(int(i), int(j)) for i, j in zip(rng.integers(0, nx, 60), rng.integers(ny - 3, ny, 60))]
    cfg = case.cfg()
    a = np.array(case.alpha_fixed)
    p1, p2, p3 = (np.ascontiguousarray(g, dtype=np.float64) for g in got)
    errs = [0.0, 0.0, 0.0]
    for i, j in pts:
        r1 = phi0[j, i] + dt * oracle.point_L(cfg, phi0, i, j, a)
        r2 = 0.75 * phi0[j, i] + 0.25 * (p1[j, i] + dt * oracle.point_L(cfg, p1, i, j, a))
        r3 = phi0[j, i] / 3.0 + 2.0 * (p2[j, i] + dt * oracle.point_L(cfg, p2, i, j, a)) / 3.0
        errs = [max(errs[0], abs(p1[j, i] - r1)), max(errs[1], abs(p2[j, i] - r2)), max(errs[2], abs(p3[j, i] - r3))]
    tol = 64 * 2.0**-24 * np.abs(phi0).max()
    assert max(errs) <= tol, (errs, tol)


def _patch_stages(phi0, i, j, dx, dt, alpha, weights):
    """The oracle's phi_1 on the 13 x 13 nodes, phi_2 on the 7 x 7 nodes and phi^{n+1} at the node
    around (i, j) of one RK3 step (Step 5) with the flux alpha `alpha` in every stage, from a 19 x 19
    periodic patch of phi0 centred on (i, j): each stage widens the dependence by three nodes, so
    the patch's own periodic wrap never reaches a node that is evaluated."""
    n = phi0.shape[0]
    rows = (j + np.arange(-9, 10)) % n
    cols = (i + np.arange(-9, 10)) % n
    p0 = np.ascontiguousarray(phi0[np.ix_(rows, cols)])
    cfg = oracle.make_cfg(dim=2, nx=19, ny=19, dx=dx, ham="burgers2d", weights=weights, alpha_mode="global_lagged")
    p1 = p0.copy()
    for b in range(3, 16):
        for a in range(3, 16):
            p1[b, a] = p0[b, a] + dt * oracle.point_L(cfg, p0, a, b, alpha)
    p2 = p1.copy()
    for b in range(6, 13):
        for a in range(6, 13):
            p2[b, a] = 0.75 * p0[b, a] + 0.25 * (p1[b, a] + dt * oracle.point_L(cfg, p1, a, b, alpha))
    p3 = p0[9, 9] / 3.0 + 2.0 * (p2[9, 9] + dt * oracle.point_L(cfg, p2, 9, 9, alpha)) / 3.0
    return p1, p2, p3


@pytest.mark.parametrize("precision,weights", [("mixed", "arclength"), ("mixed", "jp"), ("fp64", "arclength")])
def test_full_size_8192_three_stages_global_lagged(precision, weights):
    # The configuration bench.py times (Example 3 on 8192^2, lagged grid-wide alpha): all three RK
    # stages on the GPU, phi_1, phi_2 and phi^{n+1} checked at sampled nodes -- tile corners and edges,
    # the periodic seams, random interior nodes -- against the oracle's stages on patches around them.
    # Flux alpha: the grid maximum of |u + v + 1| over phi0's one-sided derivatives, which the oracle
    # evaluates on the line x + y = 1 (i + j = 10240), where |phi_x + phi_y + 1| = pi + 1 is attained;
    # later stages' maxima differ by O(dt) relative, and alpha enters L only through
    # alpha (u^+ - u^-) / 2, with |u^+ - u^-| = O(dx^5) on these smooth data.
    n = 8192
    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    phi0 = np.ascontiguousarray(inputs.phi0_negcos_diag_2d(x, x))
    cfg = oracle.make_cfg(dim=2, nx=n, ny=n, dx=dx, ham="burgers2d", weights=weights, alpha_mode="global_lagged")
    amax = 0.0
    for i in range(2049, 8192, 97):
        d = oracle.point_derivs(cfg, phi0, i, 10240 - i)
        amax = max(amax, *(abs(u + v + 1.0) for u in d[:2] for v in d[2:]))
    assert abs(amax - (1.0 + math.pi)) < 1e-9
    alpha = np.array([amax, amax])
    dt = 0.6 / (2 * amax / dx)
    case = Case(2, n, n, "burgers2d", lo=-2.0, hi=2.0, precision=precision, weights=weights,
                alpha_mode="global_lagged")
    with case.solver() as s:
        s.set_phi0(phi0)
        s.run_stage(1, dt)
        g1 = s.get_stage_phi(1)
        s.run_stage(2, dt)
        g2 = s.get_stage_phi(2)
        s.run_stage(3, dt)
        g3 = s.get_phi()
        a_gpu = s.get_state().alpha
    rng = np.random.default_rng(81920)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (63, 31), (64, 32), (8191, 4095), (4096, 8191),
           (2, 5000), (8189, 17), (3000, 8190), (1000, 2)]
    pts += [(int(i), int(j)) for i, j in rng.integers(0, n, size=(60, 2))]
    tol = (1e-12 if precision == "fp64" else 64 * 2.0**-24) * np.abs(phi0).max()
    errs = [0.0, 0.0, 0.0]
    for i, j in pts:
        p1, p2, p3 = _patch_stages(phi0, i, j, dx, dt, alpha, weights)
        rows = (j + np.arange(-6, 7)) % n
        cols = (i + np.arange(-6, 7)) % n
        errs[0] = max(errs[0], np.abs(g1[np.ix_(rows, cols)] - p1[3:16, 3:16]).max())
        rows, cols = (j + np.arange(-3, 4)) % n, (i + np.arange(-3, 4)) % n
        errs[1] = max(errs[1], np.abs(g2[np.ix_(rows, cols)] - p2[6:13, 6:13]).max())
        errs[2] = max(errs[2], abs(g3[j, i] - p3))
    assert max(errs) <= tol, (errs, tol)
    # the lagged alpha the GPU holds after stage 3 is the grid maximum over phi_2's derivatives: the
    # gradient is constant along characteristics, so it differs from phi0's maximum only by where the
    # nodes sample the moved profile, O(dt^2) relative, and never exceeds pi + 1 beyond rounding
    for a in a_gpu:
        assert abs(a - amax) <= 1e-5 * amax and a <= (1.0 + math.pi) * (1 + 1e-6), (a, amax)


@pytest.mark.parametrize("weights", ["arclength", "jp"])
def test_1d_kink_solve_matches_oracle(weights):
    # Example 6 at t = 3.5/pi^2 (kink formed) on the paper's 80-node grid, FP64
    n = 80
    x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
    case = Case(1, n, 1, "burgers1d", weights=weights, alpha_mode="default")
    phi0 = inputs.phi0_negcos_1d(x)
    tf = 3.5 / math.pi**2
    ref, steps, _, _, st = oracle.solve(case.cfg(), phi0, tf)
    with case.solver() as s:
        s.set_phi0(phi0)
        assert s.step_to(tf) == steps
        assert rel_err(s.get_phi(), ref) <= 1e-12


def test_riemann_linextrap_mixed_vs_fp64_gpu():
    # Example 10's non-convex H = sin(p+q) with linear-extrapolation boundaries on 256^2:
    # the mixed path stays within a stated distance of the FP64 path after 60 steps
    n = 256
    x, dx = inputs.axis(n, -1.0, 1.0, "linextrap")
    phi0 = inputs.phi0_riemann_2d(x, x)
    out = {}
    for prec in ("fp64", "mixed"):
        case = Case(2, n, n, "sin2d", bc="linextrap", precision=prec)
        with case.solver() as s:
            s.set_phi0(phi0)
            s.advance(60)
            s.sync()
            out[prec] = s.get_phi()
    assert np.all(np.isfinite(out["mixed"]))
    assert np.max(np.abs(out["mixed"] - out["fp64"])) < 1e-4


def _paper_table(name):
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[int(v[0])] = {"arclength": float(v[1]), "jp": float(v[3])}   # L-infinity columns
    return rows


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("ham,table", [("burgers2d", "table3_ex3_burgers2d.txt"),
                                       ("negcos2d", "table4_ex4_negcos2d.txt")])
def test_gpu_reproduces_tables_3_4(ham, table, weights):
    # FP64 GPU solves of Examples 3 and 4 with dt ~ dx^{5/3}: L-infinity errors against the exact
    # solution within 2x of the paper's Tables 3 and 4 from 40^2 to 320^2
    import exact

    tab = _paper_table(table)
    tf = 0.5 / math.pi**2
    for n in (40, 80, 160, 320):
        x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
        case = Case(2, n, n, ham, weights=weights, lo=-2.0, hi=2.0, dt_mode="dx53")
        with case.solver() as s:
            s.set_phi0(inputs.phi0_negcos_diag_2d(x, x))
            s.step_to(tf)
            e = np.abs(s.get_phi() - exact.negcos_diag_2d(ham, x, x, tf)).max()
        assert tab[n][weights] / 2 < e < tab[n][weights] * 2, (n, e, tab[n][weights])


@pytest.mark.parametrize("weights", ["arclength", "jp"])
@pytest.mark.parametrize("ham,table,tf,factor", [("advect1d", "table1_ex1_advection.txt", 2.0, 1.6),
                                                 ("negcos1d", "table2_ex2_negcos1d.txt", 0.5 / math.pi**2, 1.3)])
def test_gpu_reproduces_tables_1_2(ham, table, tf, factor, weights):
    # FP64 GPU solves of Examples 1 and 2 (node-local alpha, dt ~ dx^{5/3}): L-infinity errors against
    # the exact solution within the factors the oracle meets, from N = 20 to 320
    import exact

    tab = _paper_table(table)
    for n in (20, 40, 80, 160, 320):
        x, dx = inputs.axis(n, -1.0, 1.0, "periodic")
        case = Case(1, n, 1, ham, weights=weights, alpha_mode="local_lagged", dt_mode="dx53")
        with case.solver() as s:
            s.set_phi0(inputs.phi0_negcos_1d(x))
            s.step_to(tf)
            got = s.get_phi()
        ex = -np.cos(np.pi * (x - tf)) if ham == "advect1d" else exact.negcos_1d(ham, x, tf)
        e = np.abs(got - ex).max()
        assert tab[n][weights] / factor < e < tab[n][weights] * factor, (n, e, tab[n][weights])
