"""The no-allocation entry point against the allocating path.

alw_step_noalloc serves callers that cannot allocate device memory on demand
(a framework whose pool owns all device memory, a real-time loop that must not
allocate after start-up): it runs the same FP64 stage kernel out of a fixed
working array inside the library.  Its result must match the solver path
(alw_create / alw_set_phi0_device / alw_run_stage) within the FP64 tolerance
of the other parity tests, on two calls in a row with different grids, so that
whatever the first call leaves in the shared working array cannot leak into
the second.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpucase import Case, rel_err
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
    ]
    for case, seed, nsteps, dt in cases:
        phi0 = case.field(seed=seed)
        ref = _reference(case, phi0, dt, nsteps)
        dev_in = torch.tensor(phi0, dtype=torch.float64, device="cuda").contiguous()
        dev_out = torch.empty_like(dev_in)
        native.step_noalloc(dev_in, dev_out, dim=case.dim, nx=case.nx, ny=case.ny, bc=case.bc, xlo=case.lo,
                            xhi=case.hi, ylo=case.lo, yhi=case.hi, ham=case.ham, weights=case.weights,
                            alpha_mode=case.alpha_mode, dt=dt, nsteps=nsteps)
        got = dev_out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref) <= FP64_TOL


def test_noalloc_rejects_grids_beyond_its_storage():
    import torch

    native.load()
    n = 1024
    dev = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    with pytest.raises(native.AlwError) as ei:
        native.step_noalloc(dev, dev, dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                            dt=1e-4, nsteps=1)
    assert ei.value.status == native.EBUDGET
