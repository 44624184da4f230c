"""Whole-workload checks of the named configurations:

* bipoles40_256x256x256 (40 bipoles, solenoidal driver): FP64 and FP32 GPU
  runs of 20 full RK3 steps against the FP64 oracle, relative L2 per field
  (FP64 1e-11, FP32 1e-4);
* bipoles8_64x64x64 (the gradient workload): the B_z misfit on layer 48
  after 100 steps against a target from a forward run of another seeded
  8-bipole magnetogram; its gradient with respect to (B_z, v0, v1), B_z
  being both the nudging target and the source of the initial potential
  field, through the adjoint against central differences along 10 random
  directions (FP64 1e-6, FP32 1e-3);
* a 16^3 box: every component of the gradient of a photospheric B_z misfit
  against central differences of the FP64 oracle.
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


def _T(a, prec):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == 64 else torch.float32, device="cuda")


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_bipoles40_256_20_steps_against_the_oracle():
    """The bench workload at full size: 20 steps on the GPU in FP64 and FP32
    and in the oracle (about 3 minutes of 16 host cores)."""
    from paper_1908_08557_gb300 import Simulation
    case = inputs.make_case("bipoles40_256x256x256")
    steps = 20
    got = {}
    for prec in (64, 32):
        sim = Simulation(case.params, _T(case.state, prec), case.lnrho0, case.lnT0, precision=prec)
        sim.set_driver(_T(case.bz, prec), _T(case.v0, prec), _T(case.v1, prec), case.t0, case.t1)
        sim.step(steps)
        got[prec] = (sim.read().double().cpu().numpy(), sim.time()[0])
        sim.close()
    torch.cuda.empty_cache()
    u, t, dts = oracle.run_case(case, nsteps=steps)
    ref = oracle.interior(u)
    del u
    for prec, tol in ((64, 1e-11), (32, 1e-4)):
        g, tg = got[prec]
        errs = [_rel_l2(g[f], ref[f]) for f in range(8)]
        print(f"FP{prec} vs oracle after {steps} steps, rel L2 per field:", ["%.2e" % e for e in errs])
        assert max(errs) <= tol, (prec, errs)
        assert abs(tg - t) <= (1e-12 if prec == 64 else 1e-5) * t


def _gradient_case(prec_dt=0.017):
    c = inputs.make_case("bipoles8_64x64x64")
    c.params = dict(c.params, dt_fixed=prec_dt)
    return c


def _potential_field_torch(bz, nz, dx, dy, dz):
    """The initial potential field of a magnetogram (the input generator's
    spectral extension, A_z = 0), written with torch's FFT so that autograd
    carries the gradient from the initial state back to B_z."""
    ny, nx = bz.shape
    dev = bz.device
    kx = 2 * np.pi * torch.fft.rfftfreq(nx, d=dx, dtype=torch.float64, device=dev)[None, :]
    ky = 2 * np.pi * torch.fft.fftfreq(ny, d=dy, dtype=torch.float64, device=dev)[:, None]
    kk = torch.sqrt(kx ** 2 + ky ** 2)
    bh = torch.fft.rfft2(bz.double())
    keep = torch.ones_like(kk)
    keep[0, 0] = 0.0
    keep[:, nx // 2] = 0.0
    keep[ny // 2, :] = 0.0
    inv = torch.where(kk > 0, 1.0 / torch.where(kk > 0, kk, 1.0) ** 2, 0.0) * keep
    axh = 1j * ky * bh * inv
    ayh = -1j * kx * bh * inv
    z = torch.arange(nz, dtype=torch.float64, device=dev)[:, None, None] * dz
    dec = torch.exp(-kk[None] * z)
    ax = torch.fft.irfft2(axh[None] * dec, s=(ny, nx))
    ay = torch.fft.irfft2(ayh[None] * dec, s=(ny, nx))
    return torch.stack([ax, ay, torch.zeros_like(ax)])


def _state_of(case, bz):
    """The workload's initial state with A the potential field of bz."""
    st = case.state.copy()
    ax, ay, az = inputs.initial_potential_field(bz, case.params["nz"], case.params["dx"], case.params["dy"],
                                                case.params["dz"])
    st[0], st[1], st[2] = ax, ay, az
    return st


def _run_bz(case, prec, nsteps, k, bz, v0, v1):
    from paper_1908_08557_gb300 import Simulation
    st = _state_of(case, bz)
    sim = Simulation(case.params, _T(st, prec), case.lnrho0, case.lnT0, precision=prec, adjoint=True)
    sim.set_driver(_T(bz, prec), _T(v0, prec), _T(v1, prec), case.t0, case.t1)
    sim.set_time(0.0)
    sim.step(nsteps)
    b = sim.bz_plane(sim.read(), k).double().cpu().numpy()
    sim.close()
    return b


@pytest.mark.parametrize("prec,tol,eps", [(64, 1e-6, 1e-3), (32, 1e-3, 1e-1)])
def test_gradient_workload_64cube_100_steps_layer48(prec, tol, eps):
    """Configuration of the gradient workload: 64^3, 100 steps, loss
    1/2 sum (B_z(z = 48) - B_z,target)^2, the target from a forward run of a
    different seeded 8-bipole magnetogram (its potential field as initial
    state, its nudging target).  The run starts from the potential field of
    the parameter B_z, which it is also nudged toward: within 100 steps
    (t = 1.7) no signal from the photosphere crosses the cool bottom layers
    (sound speed ~1.3 over 12 cells), so layer 48 depends on B_z through the
    initial field.  The adjoint gradient (DrivenRun with the initial-state
    adjoint, BzPlane, binomial checkpointing with 10 slots, the initial
    field's spectral map by torch autograd) against central differences
    along 10 random directions in (B_z, v0, v1)."""
    from paper_1908_08557_gb300 import Simulation
    from paper_1908_08557_gb300.adjoint import BzPlane, DrivenRun
    case = _gradient_case()
    p = case.params
    nsteps, k = 100, 48
    bz_other = inputs.magnetogram_bipoles(64, 64, 8, seed=1)
    target = _run_bz(case, 64, nsteps, k, bz_other, case.v0, case.v1)

    def loss_of(bz, v0, v1):
        b = _run_bz(case, prec, nsteps, k, bz, v0, v1)
        return 0.5 * float(((b - target) ** 2).sum())

    tdt = torch.float64 if prec == 64 else torch.float32
    sim = Simulation(p, _T(case.state, prec), case.lnrho0, case.lnT0, precision=prec, adjoint=True)
    bz = torch.tensor(case.bz, dtype=torch.float64, device="cuda", requires_grad=True)
    v0 = _T(case.v0, prec).requires_grad_(True)
    v1 = _T(case.v1, prec).requires_grad_(True)
    a0 = _potential_field_torch(bz, p["nz"], p["dx"], p["dy"], p["dz"])
    rest = _T(case.state[3:], 64)
    state0 = torch.cat([a0, rest]).to(tdt)
    st = DrivenRun.apply(bz.to(tdt), v0, v1, sim, state0, nsteps, 10, case.t0, case.t1)
    b = BzPlane.apply(st, sim, k)
    loss = 0.5 * ((b.double() - _T(target, 64)) ** 2).sum()
    loss.backward()
    g = [bz.grad.double().cpu().numpy(), v0.grad.double().cpu().numpy(), v1.grad.double().cpu().numpy()]
    sim.close()
    lval = float(loss.detach())
    assert lval > 1e-6
    rng = np.random.default_rng(17)
    rel = []
    for _ in range(10):
        d = [rng.standard_normal(case.bz.shape), 0.01 * rng.standard_normal(case.v0.shape),
             0.01 * rng.standard_normal(case.v1.shape)]
        lp = loss_of(case.bz + eps * d[0], case.v0 + eps * d[1], case.v1 + eps * d[2])
        lm = loss_of(case.bz - eps * d[0], case.v0 - eps * d[1], case.v1 - eps * d[2])
        fd = (lp - lm) / (2 * eps)
        ad = float(sum(np.sum(gi * di) for gi, di in zip(g, d)))
        rel.append(abs(fd - ad) / abs(ad))
        assert abs(ad) > 1e-6 * lval
    print(f"FP{prec}: loss {lval:.6e}, FD vs adjoint relative errors:", ["%.1e" % r for r in rel])
    assert max(rel) <= tol, rel


def test_bruteforce_oracle_gradient_16cube():
    """Every component of the gradient of the B_z misfit on the photosphere
    of a 16^3 box after 3 steps (256 + 512 + 512 parameters, which act there
    through the nudging of A_hor and u_hor) against central differences of
    the FP64 CPU oracle."""
    from paper_1908_08557_gb300.adjoint import BzPlane, DrivenRun
    from paper_1908_08557_gb300 import Simulation
    c = inputs.make_box(16, 16, 16, seed=8, magnetogram="bipoles", n_mag=6)
    c.params = dict(c.params, dt_fixed=0.02)
    rng = np.random.default_rng(15)
    st0 = c.state.copy()
    st0[3:6] += 0.02 * rng.standard_normal(st0[3:6].shape)
    st0[0:3] += 0.01 * rng.standard_normal(st0[0:3].shape)
    c.state = st0
    p = c.params
    k, nsteps = 0, 3
    target = np.sin(np.arange(256).reshape(16, 16) * 0.3) * 0.1
    sim = Simulation(p, _T(c.state, 64), c.lnrho0, c.lnT0, precision=64, adjoint=True)
    bz = _T(c.bz, 64).requires_grad_(True)
    v0 = _T(c.v0, 64).requires_grad_(True)
    v1 = _T(c.v1, 64).requires_grad_(True)
    st = DrivenRun.apply(bz, v0, v1, sim, _T(c.state, 64), nsteps, 3, c.t0, c.t1)
    b = BzPlane.apply(st, sim, k)
    loss_t = 0.5 * ((b - _T(target, 64)) ** 2).sum()
    loss_t.backward()
    loss = float(loss_t.detach())
    grads = {"bz": bz.grad.cpu().numpy(), "v0": v0.grad.cpu().numpy(), "v1": v1.grad.cpu().numpy()}
    sim.close()

    def oracle_loss(bzv, v0v, v1v):
        axt, ayt = oracle.a_target(p, bzv)
        u = oracle.to_padded(c.state)
        oracle.run(p, u, c.lnrho0, axt, ayt, v0v, v1v, c.t0, c.t1, 0.0, nsteps)
        oracle.fill_ghosts(p, u, c.lnrho0)
        bb = oracle.deriv(p, u, 1, 0, 0)[k] - oracle.deriv(p, u, 0, 0, 1)[k]
        return 0.5 * float(((bb - target) ** 2).sum())

    assert abs(oracle_loss(c.bz, c.v0, c.v1) - loss) <= 1e-10 * loss
    eps = 1e-5
    scale = max(np.abs(g).max() for g in grads.values())
    assert scale > 1e-4
    base = {"bz": c.bz, "v0": c.v0, "v1": c.v1}
    for name, g in grads.items():
        fd = np.zeros_like(g)
        for idx in np.ndindex(g.shape):
            ap = {kk: vv.copy() for kk, vv in base.items()}
            am = {kk: vv.copy() for kk, vv in base.items()}
            ap[name][idx] += eps
            am[name][idx] -= eps
            fd[idx] = (oracle_loss(ap["bz"], ap["v0"], ap["v1"]) - oracle_loss(am["bz"], am["v0"], am["v1"])) / (2 * eps)
        assert np.abs(fd - g).max() <= 1e-6 * scale, (name, np.abs(fd - g).max(), scale)
