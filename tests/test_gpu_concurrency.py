"""Several handles at once: two handles on two streams stepping interleaved
without host synchronisation, and the library's first use in a process from
two host threads at the same time (the one-time per-device set-up of the
kernels -- shared-memory limits, CTA counts, FFT attributes, tensor-map
encoder -- runs once, under its lock).  Each run must equal the same run
made alone, bit for bit.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1908_08557_gb300.build import build
    build()


def _make(case, precision, stream=None):
    from paper_1908_08557_gb300 import Simulation
    dt = torch.float64 if precision == 64 else torch.float32
    T = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    sim = Simulation(case.params, T(case.state), case.lnrho0, case.lnT0, precision=precision, stream=stream,
                     stats_every=2)
    sim.set_driver(T(case.bz), T(case.v0), T(case.v1), case.t0, case.t1)
    return sim


@pytest.mark.parametrize("precision", [32, 64])
def test_two_handles_on_two_streams(precision):
    ca = inputs.make_box(64, 32, 24, seed=91, magnetogram="bipoles", n_mag=8)
    cb = inputs.make_box(32, 64, 20, seed=92, magnetogram="bipoles", n_mag=8)
    ref = []
    for c in (ca, cb):
        s = _make(c, precision)
        s.step(6)
        ref.append((s.read().clone(), s.time(), s.read_stats()))
        s.close()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a, b = _make(ca, precision, stream=sa), _make(cb, precision, stream=sb)
    for _ in range(6):
        a.step(1)
        b.step(1)
    torch.cuda.synchronize()
    for sim, (st, tm, stats) in zip((a, b), ref):
        assert torch.equal(sim.read(), st)
        assert sim.time() == tm
        assert sim.read_stats() == stats
        sim.close()


SCRIPT = r"""
import sys, threading
sys.path.insert(0, {root!r})
import torch, inputs
from paper_1908_08557_gb300 import Simulation

def run(seed, out, barrier=None):
    c = inputs.make_box(32, 32, 16, seed=seed, magnetogram="bipoles", n_mag=6)
    T = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    states = [T(c.state), T(c.bz), T(c.v0), T(c.v1)]
    torch.cuda.synchronize()
    if barrier is not None:
        barrier.wait()          # both threads make their first library call together
    with torch.cuda.stream(torch.cuda.Stream()):
        sim = Simulation(c.params, states[0], c.lnrho0, c.lnT0, precision=32)
        sim.set_driver(states[1], states[2], states[3], c.t0, c.t1)
        sim.step(5)
        out[seed] = (sim.read().cpu(), sim.time())
        sim.close()

torch.zeros(1, device="cuda")
got, barrier = {{}}, threading.Barrier(2)
th = [threading.Thread(target=run, args=(s, got, barrier)) for s in (1, 2)]
for t in th: t.start()
for t in th: t.join()
ref = {{}}
for s in (1, 2):
    run(s, ref)
ok = all(torch.equal(got[s][0], ref[s][0]) and got[s][1] == ref[s][1] for s in (1, 2))
print("same" if ok else "different")
sys.exit(0 if ok else 1)
"""


def test_first_use_from_two_threads():
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "same" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
