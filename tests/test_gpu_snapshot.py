"""mhd_write_snapshot on the GPU: var.h5 / grid.h5 of a running handle in
the paper's HDF5 layout (Sect. 5.3), read back by tests/h5read.py.

The data are the ghost-filled padded state with its backgrounds added (the
same values mhd_read_padded returns after mhd_fill_ghosts), bit for bit; the
time is the handle's; writing a snapshot between steps does not change the
run (the stepping after it equals the stepping without it, bit for bit).
"""
import numpy as np
import pytest

import h5read
import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["ax", "ay", "az", "ux", "uy", "uz", "lnrho", "lnTT"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1908_08557_gb300.build import build
    build()


def _sim(case, precision, **kw):
    from paper_1908_08557_gb300 import Simulation
    dt = torch.float64 if precision == 64 else torch.float32
    T = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    sim = Simulation(case.params, T(case.state), case.lnrho0, case.lnT0, precision=precision, **kw)
    sim.set_driver(T(case.bz), T(case.v0), T(case.v1), case.t0, case.t1)
    return sim


@pytest.mark.parametrize("precision,variant", [(64, "uniform"), (32, "uniform"), (32, "zgrid_background")])
def test_snapshot_of_a_running_handle(tmp_path, precision, variant):
    if variant == "uniform":
        case = inputs.make_box(32, 16, 12, seed=61, magnetogram="bipoles", n_mag=6)
        kw = {}
    else:
        z, _, _ = inputs.stretched_z(24, 0.5, 1.5, 12, 4)
        case = inputs.make_box(32, 16, 24, seed=62, z=z, magnetogram="bipoles", n_mag=6)
        kw = {"a_background": case.state[0:3].copy()}
    p = case.params
    sim = _sim(case, precision, **kw)
    sim.step(4)
    var, grid = tmp_path / "var.h5", tmp_path / "grid.h5"
    sim.write_snapshot(var, grid)
    t = sim.time()[0]
    f = h5read.File(var)
    assert float(f.root["time"]) == t
    # the reference: the same handle's ghost-filled padded state
    sim.fill_ghosts()
    ref = sim.read_padded(0)
    dt = np.float64 if precision == 64 else np.float32
    for q, name in enumerate(NAMES):
        a = f.root["data"][name]
        assert a.dtype == np.dtype(dt)
        assert a.shape == (p["nz"] + 6, p["ny"] + 6, p["nx"] + 6)
        assert np.array_equal(a, ref[q]), name
    assert f.root["settings"]["precision"] == (b"D" if precision == 64 else b"S")
    g = h5read.File(grid).root["grid"]
    zref = p["z"] if p.get("z") is not None else np.arange(-3, p["nz"] + 3) * p["dz"]
    assert np.array_equal(g["z"], zref)
    for k in g:
        assert np.array_equal(g[k], f.root["grid"][k]), k
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_snapshot_between_steps_leaves_the_run_unchanged(tmp_path, precision):
    case = inputs.make_box(32, 16, 12, seed=63, magnetogram="bipoles", n_mag=6)
    a = _sim(case, precision)
    b = _sim(case, precision)
    a.step(3)
    a.write_snapshot(tmp_path / "v.h5")
    a.step(3)
    b.step(6)
    assert torch.equal(a.read(), b.read())
    assert a.time() == b.time()
    a.close()
    b.close()


def test_snapshot_errors(tmp_path):
    from paper_1908_08557_gb300.binding import MHD_ERR_ARG, MHD_ERR_IO, MHDError
    case = inputs.make_box(16, 16, 8, seed=64, magnetogram="bipoles", n_mag=4)
    sim = _sim(case, 64)
    with pytest.raises(MHDError) as e:
        sim.write_snapshot(None, None)
    assert e.value.code == MHD_ERR_ARG
    with pytest.raises(MHDError) as e:
        sim.write_snapshot(tmp_path / "missing" / "v.h5")
    assert e.value.code == MHD_ERR_IO
    sim.step(1)  # the handle still steps
    sim.close()
