"""A stored as a perturbation about an FP64 background field (params
a_background, mhd_set_a_background) against the FP64 CPU oracle, which always
works on the full A.

The storage format changes no equation (every stencil is linear in A), so the
FP64 path must still agree with the oracle to rounding and the FP32 path to
its usual tolerances; with the background the FP32 rounding of A scales with
the perturbation.  The production-geometry checks (1024^2 planes, |A| of
several hundred) are in test_gpu_parity.py and test_gpu_production.py.
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


def _case(nx, ny, nz, seed, **kw):
    """A box whose A is the potential field A0 plus a small perturbation;
    returns the case (state = full A), A0 (FP64) and the perturbation."""
    case = inputs.make_box(nx, ny, nz, seed=seed, **kw)
    rng = np.random.default_rng(seed + 100)
    st = case.state.copy()
    a0 = st[0:3].copy()
    pert = 0.01 * rng.standard_normal(a0.shape)
    st[0:3] = a0 + pert
    st[3:6] += 0.05 * rng.standard_normal(st[3:6].shape)
    st[7] += 0.02 * rng.standard_normal(st[7].shape)
    case.state = st
    return case, a0, pert


def _bsim(case, precision, a0, pert=None, params=None, driver=True, stats_every=0):
    """Handle with A stored about a0: the state's A becomes a0 + pert (pert
    rounded to the handle's precision)."""
    from paper_1908_08557_gb300 import Simulation
    p = params or case.params
    dt = torch.float64 if precision == 64 else torch.float32
    sim = Simulation(p, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                     precision=precision, stats_every=stats_every, a_background=a0)
    if pert is not None:
        sim.set_a_background(a0, torch.tensor(pert, dtype=dt, device="cuda"))
    if driver:
        sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"),
                       torch.tensor(case.v0, dtype=dt, device="cuda"),
                       torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    return sim


def _full_state(case, a0, pert, precision):
    """The state the oracle sees: A = a0 + pert with pert as the handle holds
    it; the other fields as in the case, rounded like the handle's copy."""
    st = case.state.copy()
    if precision == 32:
        st = st.astype(np.float32).astype(np.float64)
        pert = pert.astype(np.float32).astype(np.float64)
    st[0:3] = a0 + pert
    return st


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("precision,shape,bcz", [(64, (16, 16, 12), 0), (64, (40, 24, 20), 1), (64, (32, 16, 10), 0),
                                                 (32, (16, 16, 12), 0), (32, (32, 16, 10), 0)])
def test_background_rhs(precision, shape, bcz):
    """Right-hand side of A = A0 + A' (ghost fill, swamp layers, nudging)
    against the oracle on the full A: FP64 to 1e-11, FP32 to 2e-4 of each
    field's scale."""
    case, a0, pert = _case(*shape, seed=31)
    p = dict(case.params, bc_z=bcz)
    sim = _bsim(case, precision, a0, pert, params=p, driver=(bcz == 0))
    sim.fill_ghosts()
    t = 0.41
    got = sim.eval_rhs(t).astype(np.float64)
    st = _full_state(case, a0, pert, precision)
    u = oracle.fill_ghosts(p, oracle.to_padded(st), case.lnrho0)
    if precision == 64:
        # the state read back (A' + A_bg, ghosts included) is the full state
        gp = sim.read_padded(0)
        for f in range(8):
            assert np.abs(gp[f] - u[f]).max() <= 1e-13 * np.abs(u[f]).max(), f
    r32 = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == 32 else (lambda a: a)
    if bcz == 0:
        # the nudging target difference is formed in FP64 from the handle's B_z
        axt, ayt = oracle.a_target(p, r32(case.bz))
        v0, v1 = r32(case.v0), r32(case.v1)
    else:
        nx, ny = shape[0], shape[1]
        axt = ayt = np.zeros((ny, nx))
        v0 = v1 = np.zeros((2, ny, nx))
    ref = oracle.rhs(p, u, axt, ayt, v0, v1, case.t0, case.t1, t)
    tol = 1e-11 if precision == 64 else 2e-4
    for f in range(8):
        s = np.abs(ref[f]).max()
        e = np.abs(got[f] - ref[f]).max()
        assert e <= tol * max(s, 1e-30), (f, e, s)


@pytest.mark.parametrize("precision,variant", [(64, "default"), (32, "default"), (32, "simple")])
def test_background_full_run_spots4_32(precision, variant, monkeypatch):
    """Workload spots4_32x32x32 (50 RK3 steps) with A stored about its initial
    potential field: FP64 within 1e-11 relative L2 per field of the oracle,
    FP32 within 1e-4 (the fused pair kernel and the one-cell-per-thread
    kernel)."""
    if variant == "simple":
        monkeypatch.setenv("MHD_RK_VARIANT", "simple")
    case = inputs.make_case("spots4_32x32x32")
    a0 = case.state[0:3].copy()
    sim = _bsim(case, precision, a0)
    sim.step(case.nsteps)
    got = sim.read().cpu().numpy().astype(np.float64)
    u, t, dts = oracle.run_case(case)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    print(precision, variant, "rel L2 per field:", ["%.2e" % e for e in errs])
    assert max(errs) <= (1e-11 if precision == 64 else 1e-4), errs
    tg, _ = sim.time()
    assert abs(tg - t) <= (1e-12 if precision == 64 else 1e-5) * t


@pytest.mark.parametrize("precision", [64, 32])
def test_background_cfl_and_stats(precision):
    """The CFL step and the diagnostics see the full B = curl A' + B_bg."""
    case, a0, pert = _case(32, 32, 16, seed=33)
    sim = _bsim(case, precision, a0, pert)
    sim.fill_ghosts()
    st = _full_state(case, a0, pert, precision)
    u = oracle.fill_ghosts(case.params, oracle.to_padded(st), case.lnrho0)
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
    bscale = np.sqrt(2.0 * ref[1] / (32 * 32 * 16)) / case.params["dx"]
    assert s["divb_max"] <= (1e-10 if precision == 64 else 1e-3) * bscale


def test_background_read_write_and_reset():
    """read() returns A' + A_bg; write() stores A - A_bg; a second
    mhd_set_a_background replaces background and perturbation."""
    case, a0, pert = _case(16, 16, 12, seed=35)
    sim = _bsim(case, 64, a0, pert)
    got = sim.read().cpu().numpy()
    assert np.allclose(got[0:3], a0 + pert, rtol=0, atol=1e-14 * np.abs(a0).max())
    assert np.array_equal(got[3:], case.state[3:])
    # the same full state under another split of background and perturbation
    b = a0 + 0.3
    sim.set_a_background(b, torch.tensor(pert - 0.3, device="cuda"))
    got2 = sim.read().cpu().numpy()
    assert np.allclose(got2[0:3], a0 + pert, rtol=0, atol=1e-13 * np.abs(a0).max())
    # write the full state back and read it again
    sim.write(torch.tensor(case.state, device="cuda"))
    got3 = sim.read().cpu().numpy()
    assert np.allclose(got3, case.state, rtol=0, atol=1e-13 * np.abs(case.state).max())
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_background_zero_is_the_plain_path(precision):
    """A zero background with the whole A as perturbation: every table is
    zero and the nudging target is the inversion itself, so three steps equal
    the handle without the option bit for bit."""
    from paper_1908_08557_gb300 import Simulation
    case, a0, pert = _case(16, 16, 12, seed=37)
    dt = torch.float64 if precision == 64 else torch.float32
    outs = []
    for abg in (False, True):
        sim = Simulation(case.params, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0, case.lnT0,
                         precision=precision, a_background=np.zeros_like(a0) if abg else None)
        if abg:
            sim.set_a_background(np.zeros_like(a0), torch.tensor(case.state[0:3], dtype=dt, device="cuda"))
        sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"), torch.tensor(case.v0, dtype=dt, device="cuda"),
                       torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
        sim.step(3)
        outs.append(sim.read())
        sim.close()
    assert torch.equal(outs[0], outs[1])


def test_background_argument_errors():
    from paper_1908_08557_gb300 import Simulation, binding
    case, a0, pert = _case(16, 16, 12, seed=39)
    sim = Simulation(case.params, torch.tensor(case.state, dtype=torch.float64, device="cuda"), case.lnrho0,
                     case.lnT0, precision=64)
    with pytest.raises(binding.MHDError) as e:
        sim.set_a_background(a0)
    assert e.value.code == binding.MHD_ERR_ARG
    sim.close()
    with pytest.raises(binding.MHDError) as e:
        Simulation(case.params, torch.tensor(case.state, dtype=torch.float64, device="cuda"), case.lnrho0,
                   case.lnT0, precision=64, adjoint=True, a_background=a0)
    assert e.value.code == binding.MHD_ERR_ARG
