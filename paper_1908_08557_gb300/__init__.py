"""GB300-native driven coronal MHD step (Bourdin 2019): CUDA library libmhd
(sm_103a) behind a C ABI, with a thin Python binding.

    from paper_1908_08557_gb300 import build, Simulation
    build()                      # compile libmhd.so in-tree (nvcc)
    sim = Simulation(params, state, lnrho0, precision=32)
    sim.set_driver(bz, v0, v1, t0, t1)
    sim.step(10)
"""
from .binding import MHDError, Simulation, load, workspace_bytes  # noqa: F401
from .granulation import Granulation  # noqa: F401
from .build import build  # noqa: F401
