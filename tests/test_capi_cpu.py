"""Host-side checks that need no GPU: the CUDA library builds for sm_103a, loads,
exports every symbol include/alweno.h declares, and refuses to run without a
device instead of falling back to the CPU."""
import ctypes
import os

import numpy as np
import pytest

from paper_1909_13263_gb300 import build, native


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native.load()


def test_header_declares_the_boundary():
    names = native.header_functions()
    for required in ("alw_create", "alw_destroy", "alw_set_phi0", "alw_set_phi0_device", "alw_step_to",
                     "alw_get_phi", "alw_get_state", "alw_set_state", "alw_last_error", "alw_step_noalloc"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in native.header_functions():
        assert hasattr(lib, name), name


def test_no_cpu_fallback_without_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(native.AlwError) as e:
        native.Solver(dim=2, nx=16, ny=16, xlo=0.0, xhi=1.0, ylo=0.0, yhi=1.0, ham="burgers2d")
    assert e.value.status == native.ECUDA


def test_library_is_built_for_sm_103a(lib):
    # the build passes exactly one -gencode for compute_103a / sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(native.LIB_PATH) > 0


def test_result_buffer_argument_is_checked():
    # get_phi(out=...) writes into the caller's array only when it can take the result unchanged
    a = np.zeros((3, 4))
    assert native._host_out(a, (3, 4)) is a
    assert native._host_out(None, (3, 4)).shape == (3, 4)
    for bad in (np.zeros((4, 3)), np.zeros((3, 4), dtype=np.float32), np.zeros((4, 3)).T, [[0.0] * 4] * 3):
        with pytest.raises(ValueError):
            native._host_out(bad, (3, 4))
    ro = np.zeros((3, 4))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        native._host_out(ro, (3, 4))
