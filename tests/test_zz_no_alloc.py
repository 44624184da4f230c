"""The allocation-free magnetogram inversion (mhd_invert_magnetogram_static)
against the workspace-based path (mhd_set_driver + mhd_read_target).

The entry point exists for callers that cannot allocate device memory (a
host application that reserves the whole GPU, a plugin behind a full caching
allocator, allocation-free critical paths): its FFT scratch is a fixed
__device__ array shared by all calls.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1908_08557_gb300.build import build
    from paper_1908_08557_gb300 import binding
    build()
    return binding.load()


def _handle_target(case, precision):
    from paper_1908_08557_gb300 import Simulation
    dt = torch.float64 if precision == 64 else torch.float32
    sim = Simulation(case.params, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                     precision=precision)
    sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"), torch.tensor(case.v0, dtype=dt, device="cuda"),
                   torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    out = sim.read_target()
    sim.close()
    return out


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("shape", [(64, 32), (512, 512)])
def test_static_inversion_matches_workspace_path(lib, precision, shape):
    nx, ny = shape
    dt = torch.float64 if precision == 64 else torch.float32
    tol = 1e-13 if precision == 64 else 1e-6
    stream = torch.cuda.current_stream()
    # two calls in a row with different magnetograms: the second must not see
    # anything the first left in the shared scratch
    for seed in (21, 22):
        case = inputs.make_box(nx, ny, 8, seed=seed, dy=1.5, n_mag=6)
        ref = _handle_target(case, precision)
        bz = torch.tensor(case.bz, dtype=dt, device="cuda")
        ax = torch.full((ny, nx), float("nan"), dtype=dt, device="cuda")
        ay = torch.full((ny, nx), float("nan"), dtype=dt, device="cuda")
        rc = lib.mhd_invert_magnetogram_static(nx, ny, case.params["dx"], case.params["dy"], precision,
                                               ctypes.c_void_p(bz.data_ptr()), ctypes.c_void_p(ax.data_ptr()),
                                               ctypes.c_void_p(ay.data_ptr()),
                                               ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.mhd_last_error(None)
        torch.cuda.synchronize()
        got = np.stack([ax.cpu().numpy(), ay.cpu().numpy()]).astype(np.float64)
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol * scale


def test_static_inversion_takes_no_device_memory_after_the_first_call(lib):
    """The first call on a device loads the module that holds the scratch
    array (lazy module loading); every later call must leave the device's free
    memory exactly as it was."""
    nx = ny = 256
    bz = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    bz[10, 20], bz[200, 100] = 1.0, -1.0
    ax = torch.empty_like(bz)
    ay = torch.empty_like(bz)
    stream = torch.cuda.current_stream()
    args = (nx, ny, 1.0, 1.0, 32, ctypes.c_void_p(bz.data_ptr()), ctypes.c_void_p(ax.data_ptr()),
            ctypes.c_void_p(ay.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert lib.mhd_invert_magnetogram_static(*args) == 0, lib.mhd_last_error(None)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.mhd_invert_magnetogram_static(*args) == 0, lib.mhd_last_error(None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_inversion_rejects_oversize(lib):
    from paper_1908_08557_gb300 import binding
    rc = lib.mhd_invert_magnetogram_static(1024, 1024, 1.0, 1.0, 32, ctypes.c_void_p(256), ctypes.c_void_p(256),
                                           ctypes.c_void_p(256), None)
    assert rc == binding.MHD_ERR_ARG
    assert b"[8, 512]" in lib.mhd_last_error(None)
