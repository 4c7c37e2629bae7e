"""The no-allocation entry point against the oracle and the allocating path.

alw_step_noalloc serves callers that cannot allocate device memory on demand
(a framework whose pool owns all device memory, a real-time loop that must not
allocate after start-up): it runs the same FP64 stage kernel out of a fixed
working array inside the library.  Its result must match the FP64 oracle and
the solver path (alw_create / alw_set_phi0_device / alw_run_stage) within the
FP64 tolerance of the other parity tests, on calls in a row with different
grids, so that whatever one call leaves in the shared working array cannot
leak into the next.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpucase import Case, oracle_steps, rel_err
from paper_1909_13263_gb300 import native

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _reference(case, phi0, dt, nsteps):
    with case.solver() as s:
        s.set_phi0(phi0)
        for _ in range(nsteps):
            for stage in (1, 2, 3):
                s.run_stage(stage, dt)
        return s.get_phi()


def test_noalloc_matches_solver_path_two_calls():
    import torch

    native.load()
    cases = [
        (Case(2, 70, 37, "burgers2d", weights="arclength"), 7, 3, 2.0e-3),
        (Case(2, 40, 64, "negcos2d", bc="linextrap", weights="jp", alpha_mode="local_lagged"), 11, 2, 2.5e-3),
        (Case(1, 100, 1, "burgers1d", alpha_mode="local_lagged"), 5, 4, 1.5e-3),
        (Case(2, 33, 50, "sin2d", weights="arclength", alpha_mode="global_exact"), 3, 2, 2.0e-3),
    ]
    for case, seed, nsteps, dt in cases:
        # rough data in 2D; smooth data in 1D, where the fixed dt must stay below the CFL limit of
        # (phi_x + 1)^2 / 2 (an unstable run would amplify rounding differences without bound)
        phi0 = case.field(seed=seed, kind="smooth" if case.dim == 1 else "rough")
        ref = _reference(case, phi0, dt, nsteps)
        want = oracle_steps(case, phi0, dt, nsteps)
        dev_in = torch.tensor(phi0, dtype=torch.float64, device="cuda").contiguous()
        dev_out = torch.empty_like(dev_in)
        native.step_noalloc(dev_in, dev_out, dim=case.dim, nx=case.nx, ny=case.ny, bc=case.bc, xlo=case.lo,
                            xhi=case.hi, ylo=case.lo, yhi=case.hi, ham=case.ham, weights=case.weights,
                            alpha_mode=case.alpha_mode, dt=dt, nsteps=nsteps)
        got = dev_out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, want) <= FP64_TOL, (case, rel_err(got, want))
        assert rel_err(got, ref) <= FP64_TOL


def test_noalloc_zero_steps_returns_its_input():
    import torch

    native.load()
    case = Case(2, 45, 29, "burgers2d", bc="linextrap")
    phi0 = case.field(seed=2)
    dev_in = torch.tensor(phi0, dtype=torch.float64, device="cuda").contiguous()
    dev_out = torch.full_like(dev_in, float("nan"))
    native.step_noalloc(dev_in, dev_out, dim=2, nx=case.nx, ny=case.ny, bc=case.bc, xlo=case.lo, xhi=case.hi,
                        ylo=case.lo, yhi=case.hi, ham=case.ham, dt=1e-3, nsteps=0)
    assert np.array_equal(dev_out.cpu().numpy(), phi0)


def test_noalloc_rejects_grids_beyond_its_storage():
    import torch

    native.load()
    n = 1024
    dev = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    with pytest.raises(native.AlwError) as ei:
        native.step_noalloc(dev, dev, dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                            dt=1e-4, nsteps=1)
    assert ei.value.status == native.EBUDGET
