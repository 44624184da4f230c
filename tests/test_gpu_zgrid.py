"""Non-uniform vertical grid (Sect. 1: spacing growing with height; Sect. 4.1
Eq. 14 and Sect. 4.2 Eq. 17 with the layer distances; Sect. 5.3 dz_1) on the
GPU against the FP64 oracle on the same positions (params z).

The layer index is the uniform coordinate; every z derivative follows by the
chain rule from the sixth-order stencils of the positions, the ghost rules
and the potential-field extrapolations take the layer distances, the CFL
rule the local spacing and the diagnostics the cell extents.  Grid: spacing
from 0.5 at the photosphere to 1.5 at the top (ratio 3) around layer 12.
"""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NG = oracle.NG


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1908_08557_gb300.build import build
    build()
    oracle.build()


def _zcase(nx, ny, nz, seed, perturb=True, **kw):
    z, _, _ = inputs.stretched_z(nz, 0.5, 1.5, 12, 4)
    case = inputs.make_box(nx, ny, nz, seed=seed, z=z, magnetogram="bipoles", n_mag=6, **kw)
    if perturb:
        rng = np.random.default_rng(seed + 100)
        st = case.state.copy()
        st[3:6] += 0.05 * rng.standard_normal(st[3:6].shape)
        st[7] += 0.02 * rng.standard_normal(st[7].shape)
        st[0:3] += 0.01 * rng.standard_normal(st[0:3].shape)
        case.state = st
    return case


def _sim(case, precision, params=None, driver=True, stats_every=0):
    from paper_1908_08557_gb300 import Simulation
    p = params or case.params
    dt = torch.float64 if precision == 64 else torch.float32
    sim = Simulation(p, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                     precision=precision, stats_every=stats_every)
    if driver:
        sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"), torch.tensor(case.v0, dtype=dt, device="cuda"),
                       torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    return sim


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("shape", [(16, 16, 24), (32, 16, 30)])
def test_zgrid_ghost_fill_fp64(shape):
    """Bottom Eq. 8 with the local spacing, top Eq. 13 with the distances
    z_{nz-1+m} - z_{nz-1-m}, the potential-field ghosts over the layer
    distances (both directions)."""
    case = _zcase(*shape, seed=41)
    sim = _sim(case, 64)
    sim.fill_ghosts()
    got = sim.read_padded(0)
    u = oracle.fill_ghosts(case.params, oracle.to_padded(case.state), case.lnrho0)
    for f in range(8):
        scale = np.abs(u[f]).max()
        assert np.abs(got[f] - u[f]).max() <= 1e-13 * scale, f


@pytest.mark.parametrize("precision,variant", [(64, "default"), (32, "default"), (32, "simple")])
def test_zgrid_rhs(precision, variant, monkeypatch):
    """Right-hand side on the stretched grid (chain-rule z derivatives, the
    mixed derivatives with the metric, swamp and nudging rows): FP64 to
    1e-11, FP32 to 2e-4 of each field's scale; FP32 by the fused pair kernel
    and by the one-cell-per-thread kernel."""
    if variant == "simple":
        monkeypatch.setenv("MHD_RK_VARIANT", "simple")
    case = _zcase(16, 16, 24, seed=43)
    sim = _sim(case, precision)
    sim.fill_ghosts()
    t = 0.33
    got = sim.eval_rhs(t).astype(np.float64)
    u = sim.read_padded(0).astype(np.float64)
    r32 = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == 32 else (lambda a: a)
    axt, ayt = (r32(x) for x in oracle.a_target(case.params, case.bz))
    ref = oracle.rhs(case.params, u, axt, ayt, r32(case.v0), r32(case.v1), case.t0, case.t1, t)
    tol = 1e-11 if precision == 64 else 2e-4
    for f in range(8):
        s = np.abs(ref[f]).max()
        e = np.abs(got[f] - ref[f]).max()
        assert e <= tol * max(s, 1e-30), (f, e, s)


@pytest.mark.parametrize("precision", [64, 32])
def test_zgrid_cfl_and_stats(precision):
    """CFL step with the local spacing; energies and mass with the cell
    extents; div B with the metric."""
    case = _zcase(32, 32, 24, seed=45)
    sim = _sim(case, precision)
    sim.fill_ghosts()
    u = np.ascontiguousarray(sim.read_padded(0), dtype=np.float64)
    tol = 1e-12 if precision == 64 else 1e-5
    dt = sim.compute_dt()
    assert abs(dt - oracle.cfl(case.params, u)) <= tol * dt
    s = sim.compute_stats()
    ref = oracle.stats(case.params, u)
    keys = ["e_kin", "e_mag", "e_th", "mass", "flux_net", "flux_abs", "divb_max"]
    for k in ("e_kin", "e_mag", "e_th", "mass", "flux_abs"):
        r = ref[keys.index(k)]
        assert abs(s[k] - r) <= tol * abs(r), (k, s[k], r)
    assert abs(s["flux_net"] - ref[4]) <= tol * ref[5]
    assert s["divb_max"] <= (1e-10 if precision == 64 else 1e-3) * np.sqrt(2 * ref[1] / ref[3])


@pytest.mark.parametrize("precision,variant", [(64, "default"), (32, "default"), (32, "simple")])
def test_zgrid_full_run(precision, variant, monkeypatch):
    """50 RK3 steps on the stretched grid from the stratified potential-field
    state, driven: FP64 within 1e-11, FP32 within 1e-4 relative L2 per field
    of the oracle, same time."""
    if variant == "simple":
        monkeypatch.setenv("MHD_RK_VARIANT", "simple")
    case = _zcase(32, 16, 24, seed=47, perturb=False)
    sim = _sim(case, precision)
    sim.step(50)
    got = sim.read().cpu().numpy().astype(np.float64)
    u, t, dts = oracle.run_case(case, nsteps=50)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    print(precision, variant, "zgrid rel L2 per field:", ["%.2e" % e for e in errs])
    assert max(errs) <= (1e-11 if precision == 64 else 1e-4), errs
    tg, _ = sim.time()
    assert abs(tg - t) <= (1e-12 if precision == 64 else 1e-5) * t


@pytest.mark.parametrize("precision", [64, 32])
def test_zgrid_with_a_background_rhs(precision):
    """A stored about an FP64 background on the stretched grid: the
    background's B, J, lap A and div A carry the same chain-rule metric as
    the kernels' stencils.  Right-hand side of A0 + A' against the oracle on
    the full A (FP64 1e-11, FP32 2e-4 of each field's scale)."""
    case = _zcase(16, 16, 24, seed=53)
    rng = np.random.default_rng(153)
    a0 = case.state[0:3].copy()
    pert = 0.01 * rng.standard_normal(a0.shape)
    dt = torch.float64 if precision == 64 else torch.float32
    from paper_1908_08557_gb300 import Simulation
    sim = Simulation(case.params, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                     precision=precision, a_background=a0)
    sim.set_a_background(a0, torch.tensor(pert, dtype=dt, device="cuda"))
    sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"), torch.tensor(case.v0, dtype=dt, device="cuda"),
                   torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    sim.fill_ghosts()
    t = 0.29
    got = sim.eval_rhs(t).astype(np.float64)
    r32 = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == 32 else (lambda a: a)
    st = r32(case.state.copy())
    st[0:3] = a0 + r32(pert)
    u = oracle.fill_ghosts(case.params, oracle.to_padded(st), case.lnrho0)
    axt, ayt = oracle.a_target(case.params, r32(case.bz))
    ref = oracle.rhs(case.params, u, axt, ayt, r32(case.v0), r32(case.v1), case.t0, case.t1, t)
    tol = 1e-11 if precision == 64 else 2e-4
    for f in range(8):
        s = np.abs(ref[f]).max()
        e = np.abs(got[f] - ref[f]).max()
        assert e <= tol * max(s, 1e-30), (f, e, s)


@pytest.mark.parametrize("precision", [64, 32])
def test_zgrid_with_a_background_full_run(precision):
    """50 driven steps on the stretched grid with A stored about its initial
    potential field: FP64 within 1e-11, FP32 within 1e-4 relative L2 per
    field of the oracle."""
    from paper_1908_08557_gb300 import Simulation
    case = _zcase(32, 16, 24, seed=47, perturb=False)
    dt = torch.float64 if precision == 64 else torch.float32
    sim = Simulation(case.params, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                     precision=precision, a_background=case.state[0:3].copy())
    sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"), torch.tensor(case.v0, dtype=dt, device="cuda"),
                   torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    sim.step(50)
    got = sim.read().cpu().numpy().astype(np.float64)
    u, t, dts = oracle.run_case(case, nsteps=50)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    print(precision, "zgrid + background rel L2 per field:", ["%.2e" % e for e in errs])
    assert max(errs) <= (1e-11 if precision == 64 else 1e-4), errs


def test_uniform_positions_reproduce_the_uniform_grid():
    """Positions k dz given explicitly: the same steps as the handle without
    them (FP64, to rounding; the extrapolation multipliers are then
    exp(-|k| m dz) instead of powers of exp(-|k| dz))."""
    case = inputs.make_box(16, 16, 12, seed=49, magnetogram="bipoles", n_mag=6)
    pz = dict(case.params, z=np.arange(-NG, 12 + NG) * case.params["dz"])
    a = _sim(case, 64)
    b = _sim(case, 64, params=pz)
    a.step(10)
    b.step(10)
    ga, gb = a.read().cpu().numpy(), b.read().cpu().numpy()
    for f in range(8):
        assert _rel_l2(gb[f], ga[f]) <= 1e-13, f
    assert abs(a.time()[0] - b.time()[0]) <= 1e-14 * a.time()[0]


def test_zgrid_argument_errors():
    from paper_1908_08557_gb300 import MHDError, Simulation
    from paper_1908_08557_gb300.binding import MHD_ERR_ARG, MHD_ERR_UNSUPPORTED
    case = _zcase(16, 16, 24, seed=51)
    bad = dict(case.params, z=case.params["z"][::-1].copy())
    with pytest.raises(MHDError) as e:
        Simulation(bad, torch.tensor(case.state, device="cuda"), case.lnrho0, case.lnT0, precision=64)
    assert e.value.code == MHD_ERR_ARG
    with pytest.raises(MHDError) as e:
        Simulation(case.params, torch.tensor(case.state, device="cuda"), case.lnrho0, case.lnT0, precision=64,
                   adjoint=True)
    assert e.value.code == MHD_ERR_ARG
