"""Failure detection without a GPU fault: a bounded device wait that runs out.

The fused FP32 kernel waits for each state plane's TMA copy on an mbarrier
with a bounded number of polls.  The test hook mhd_debug_skip_copy makes one
CTA not issue one copy (nor its barrier arrival), so its wait finds nothing in
flight and gives up; the kernel drains its other copies, frees its tensor
memory and records the time-out, the rest of the step returns without work,
and the host sees MHD_ERR_TIMEOUT.  Writing a state clears the flag, and the
handle then steps exactly like a fresh one.
"""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1908_08557_gb300.build import build
    build()


def _sim(case, precision):
    from paper_1908_08557_gb300 import Simulation
    dt = torch.float64 if precision == 64 else torch.float32
    sim = Simulation(case.params, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                     precision=precision)
    sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"), torch.tensor(case.v0, dtype=dt, device="cuda"),
                   torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    return sim


@pytest.mark.parametrize("plane", [-3, 1])
def test_bounded_wait_times_out_and_the_handle_recovers(plane):
    from paper_1908_08557_gb300 import MHDError
    from paper_1908_08557_gb300.binding import MHD_ERR_TIMEOUT
    case = inputs.make_box(64, 32, 20, seed=21)
    sim = _sim(case, 32)
    # plane -3 is the first copy of the first z chunk; plane 1 a later one,
    # waited for while other copies are in flight
    sim.debug_skip_copy(plane, 1 << 16)
    sim.step(1)
    with pytest.raises(MHDError) as e:
        sim.time()
    assert e.value.code == MHD_ERR_TIMEOUT
    # further steps are no-ops while the flag is set
    sim.step(1)
    with pytest.raises(MHDError):
        sim.time()
    # a fresh state clears the flag; the handle then steps like a new one
    sim.write(torch.tensor(case.state, dtype=torch.float32, device="cuda"))
    sim.set_time(0.0)
    sim.step(2)
    ref = _sim(case, 32)
    ref.step(2)
    assert torch.equal(sim.read(), ref.read())
    assert sim.time() == ref.time()
    sim.close()
    ref.close()


def test_hook_argument_errors():
    from paper_1908_08557_gb300 import MHDError
    from paper_1908_08557_gb300.binding import MHD_ERR_ARG, MHD_ERR_UNSUPPORTED
    case = inputs.make_box(16, 16, 10, seed=22)
    sim = _sim(case, 64)
    with pytest.raises(MHDError) as e:
        sim.debug_skip_copy(0, 100)
    assert e.value.code == MHD_ERR_UNSUPPORTED
    sim.close()
    sim = _sim(case, 32)
    for plane, lim in ((-4, 100), (13, 100), (0, 0)):
        with pytest.raises(MHDError) as e:
            sim.debug_skip_copy(plane, lim)
        assert e.value.code == MHD_ERR_ARG
    sim.close()
