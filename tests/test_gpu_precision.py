"""Stated precision bounds of the float paths against FP64 (Example 3, exact solution)."""
import math

import numpy as np
import pytest

import exact
from paper_1909_13263_gb300 import inputs, native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    native.load()
    native.use_torch_allocator(True)
    yield


def _solve(n, precision):
    x, dx = inputs.axis(n, -2.0, 2.0, "periodic")
    tf = 0.5 / math.pi**2
    with native.Solver(dim=2, nx=n, ny=n, xlo=-2.0, xhi=2.0, ylo=-2.0, yhi=2.0, ham="burgers2d",
                       precision=precision) as s:
        s.set_phi0(inputs.phi0_negcos_diag_2d(x, x))
        s.step_to(tf)
        return np.abs(s.get_phi() - exact.negcos_diag_2d("burgers2d", x, x, tf)).mean()


@pytest.mark.parametrize("n", [80, 160])
def test_mixed_l1_within_105_percent_of_fp64_where_discretisation_dominates(n):
    e64, emx = _solve(n, "fp64"), _solve(n, "mixed")
    assert emx <= 1.05 * e64, (emx, e64)


def test_mixed_beats_fp32_by_orders_of_magnitude_on_fine_grids():
    e64, emx, e32 = _solve(400, "fp64"), _solve(400, "mixed"), _solve(400, "fp32")
    assert emx < 2.0 * e64 and e32 > 20.0 * emx, (e64, emx, e32)
