"""Production size (workload ar_1024x1024x256: 1024 x 1024 x 256 cells,
horizontal spacing 4x vertical, 400 bipoles plus a +-5 active-region pair of
sigma = 40 cells): full RK3 steps of the FP32 path, with A stored about the
FP64 initial potential field, against an FP64 GPU run of the same steps from
the same state.  The FP64 path itself is checked against the oracle cell by
cell at this geometry (test_gpu_parity.py) and over whole runs on smaller
boxes; at this size the oracle would take hours per step.

Tolerance: 1e-4 relative L2 per field after 50 steps, the FP32 target.  The
driver is re-seeded after 25 steps (new snapshot pair, as the production run
does every 50), which also re-forms the nudging target relative to the
background.
"""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["A_x", "A_y", "A_z", "u_x", "u_y", "u_z", "ln_rho", "ln_T"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1908_08557_gb300.build import build
    build()


def _run(c, prec, steps, reseed, a_background):
    from paper_1908_08557_gb300 import Simulation
    p = c.params
    dev = torch.device("cuda:0")
    tdt = torch.float32 if prec == 32 else torch.float64
    a0 = torch.tensor(c.state[0:3], dtype=torch.float64, device=dev) if a_background else None
    sim = Simulation(p, torch.tensor(c.state, dtype=tdt, device=dev), c.lnrho0, c.lnT0, precision=prec,
                     a_background=a0)
    del a0
    bz = torch.tensor(c.bz, dtype=tdt, device=dev)
    sim.set_driver(bz, torch.tensor(c.v0, dtype=tdt, device=dev), torch.tensor(c.v1, dtype=tdt, device=dev),
                   c.t0, c.t1)
    km = min(32, p["nx"] // 2, p["ny"] // 2)
    sim.step(reseed)
    t, dt = sim.time()
    v2 = inputs.driver_solenoidal(p["nx"], p["ny"], km, 0.01, 2)
    sim.set_driver(bz, torch.tensor(c.v1, dtype=tdt, device=dev), torch.tensor(v2, dtype=tdt, device=dev),
                   t, t + reseed * dt)
    sim.step(steps - reseed)
    out = sim.read().to(torch.float64)
    t_end = sim.time()[0]
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out, t_end


def test_production_fp32_matches_fp64_50_steps():
    c = inputs.make_case("ar_1024x1024x256")
    assert np.abs(c.state[0:3]).max() > 100.0  # the regime the background storage is for
    steps, reseed = 50, 25
    ref, t64 = _run(c, 64, steps, reseed, False)
    got, t32 = _run(c, 32, steps, reseed, True)
    err = [float(torch.linalg.vector_norm(got[f] - ref[f]) / torch.linalg.vector_norm(ref[f])) for f in range(8)]
    del got
    torch.cuda.empty_cache()
    # for the record: the same FP32 run with A stored whole
    plain, _ = _run(c, 32, steps, reseed, False)
    err_plain = [float(torch.linalg.vector_norm(plain[f] - ref[f]) / torch.linalg.vector_norm(ref[f]))
                 for f in range(8)]
    del plain, ref
    torch.cuda.empty_cache()
    print("FP32 (A about the initial field) vs FP64, rel L2:", {n: "%.2e" % e for n, e in zip(NAMES, err)})
    print("FP32 (A stored whole) vs FP64, rel L2:         ", {n: "%.2e" % e for n, e in zip(NAMES, err_plain)})
    assert abs(t32 - t64) <= 1e-5 * t64
    assert max(err) <= 1e-4, dict(zip(NAMES, err))
