"""Adjoint of the RK step (frozen dt) through the C ABI: dot-product test
against central differences of the forward step, finite-difference checks of
a misfit loss through the torch.autograd.Function, bitwise independence from
the checkpoint budget, and the brute-force oracle gradient (central
differences of the FP64 oracle over every parameter) on an 8^3 box."""
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


def _case(nx, ny, nz, seed, dt=0.01, **kw):
    c = inputs.make_box(nx, ny, nz, seed=seed, magnetogram="bipoles", n_mag=6, **kw)
    c.params = dict(c.params, dt_fixed=dt)
    rng = np.random.default_rng(seed + 7)
    st = c.state.copy()
    st[3:6] += 0.02 * rng.standard_normal(st[3:6].shape)
    st[0:3] += 0.01 * rng.standard_normal(st[0:3].shape)
    st[7] += 0.01 * rng.standard_normal(st[7].shape)
    c.state = st
    return c


def _sim(case, prec):
    from paper_1908_08557_gb300 import Simulation
    return Simulation(case.params, case.state.astype(np.float64 if prec == 64 else np.float32), case.lnrho0,
                      case.lnT0, precision=prec, adjoint=True)


def _T(a, prec):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == 64 else torch.float32, device="cuda")


NC = dict(nc_tau=0.5, nc_z_max=8.0, nc_z_width=3.0)


def _cooling(case, seed):
    """Newtonian cooling on (Sect. 3.1), ln rho perturbed so the inverse
    lookup interpolates between layers."""
    rng = np.random.default_rng(seed + 11)
    case.state = case.state.copy()
    case.state[6] += 0.05 * rng.standard_normal(case.state[6].shape)
    case.params = dict(case.params, **NC)
    return case


@pytest.mark.parametrize("cooling", [False, True])
def test_one_step_dot_product_fp64(cooling):
    """<lam, (F(x + e v) - F(x - e v)) / 2e> = <J^T lam, v> for directions in
    the state and in every parameter (B_z, v0, v1); with and without the
    Newtonian cooling term."""
    case = _case(16, 16, 12, seed=1)
    if cooling:
        case = _cooling(case, 1)
    sim = _sim(case, 64)
    rng = np.random.default_rng(3)
    nz, ny, nx = 12, 16, 16
    lam = rng.standard_normal((8, nz, ny, nx))
    dx = rng.standard_normal((8, nz, ny, nx)) * 0.01
    dbz = rng.standard_normal((ny, nx)) * 0.05
    dv0 = rng.standard_normal((2, ny, nx)) * 0.01
    dv1 = rng.standard_normal((2, ny, nx)) * 0.01
    t_start = 0.3  # inside the switch-on ramp and between the driver snapshots

    def F(state, bz, v0, v1):
        sim.set_driver(_T(bz, 64), _T(v0, 64), _T(v1, 64), case.t0, case.t1)
        sim.write(_T(state, 64))
        sim.set_time(t_start)
        sim.step(1)
        return sim.read().cpu().numpy()

    eps = 1e-5
    jv = (F(case.state + eps * dx, case.bz + eps * dbz, case.v0 + eps * dv0, case.v1 + eps * dv1) -
          F(case.state - eps * dx, case.bz - eps * dbz, case.v0 - eps * dv0, case.v1 - eps * dv1)) / (2 * eps)
    lhs = float(np.sum(lam * jv))
    sim.set_driver(_T(case.bz, 64), _T(case.v0, 64), _T(case.v1, 64), case.t0, case.t1)
    sim.write(_T(case.state, 64))
    sim.set_time(t_start)
    ck = sim.new_checkpoint()
    t = sim.save(ck)
    sim.adjoint_init(_T(lam, 64))
    sim.restore(ck, t)
    sim.adjoint_step()
    g = sim.adjoint_read()
    rhs = float(np.sum(g["lam"].cpu().numpy() * dx) + np.sum(g["bz"].cpu().numpy() * dbz) +
                np.sum(g["v0"].cpu().numpy() * dv0) + np.sum(g["v1"].cpu().numpy() * dv1))
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs), (lhs, rhs)
    # each parameter block separately
    for name, d in (("bz", dbz), ("v0", dv0), ("v1", dv1)):
        args = [case.state, case.bz, case.v0, case.v1]
        idx = {"bz": 1, "v0": 2, "v1": 3}[name]
        ap = list(args); am = list(args)
        ap[idx] = args[idx] + eps * d
        am[idx] = args[idx] - eps * d
        l1 = float(np.sum(lam * (F(*ap) - F(*am)) / (2 * eps)))
        r1 = float(np.sum(g[name].cpu().numpy() * d))
        # the blocks are 1e-4 of the full product; with the cooling term's
        # ln T, ln rho coupling the central differences of the driven layers
        # carry ~1e-10 of rounding (1e-16 x values ~ 1e2 / 2e-5 per cell)
        assert abs(l1 - r1) <= (1e-5 if cooling else 1e-6) * max(abs(l1), 1e-12), (name, l1, r1)


def test_cooling_adjoint_fp32_matches_fp64():
    """One adjoint step with Newtonian cooling on: the FP32 path (pair point
    kernel, the term per lane) against the FP64 path (scalar point kernel)
    on the same state and output adjoint."""
    case = _cooling(_case(32, 16, 12, seed=4), 4)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal((8, 12, 16, 32))
    out = {}
    for prec in (64, 32):
        sim = _sim(case, prec)
        sim.set_driver(_T(case.bz, prec), _T(case.v0, prec), _T(case.v1, prec), case.t0, case.t1)
        sim.write(_T(case.state, prec))
        sim.set_time(0.3)
        ck = sim.new_checkpoint()
        t = sim.save(ck)
        sim.adjoint_init(_T(lam, prec))
        sim.restore(ck, t)
        sim.adjoint_step()
        g = sim.adjoint_read()
        out[prec] = {k: v.double().cpu().numpy() for k, v in g.items()}
        sim.close()
    for k in ("lam", "bz", "v0", "v1"):
        a, b = out[32][k], out[64][k]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), k


def _loss_and_grads(case, prec, nsteps, k, target, slots):
    from paper_1908_08557_gb300.adjoint import BzPlane, DrivenRun
    sim = _sim(case, prec)
    bz = _T(case.bz, prec).requires_grad_(True)
    v0 = _T(case.v0, prec).requires_grad_(True)
    v1 = _T(case.v1, prec).requires_grad_(True)
    st = DrivenRun.apply(bz, v0, v1, sim, _T(case.state, prec), nsteps, slots, case.t0, case.t1)
    b = BzPlane.apply(st, sim, k)
    loss = 0.5 * ((b - _T(target, prec)) ** 2).sum()
    loss.backward()
    out = (float(loss.detach()), bz.grad.double().cpu().numpy(), v0.grad.double().cpu().numpy(), v1.grad.double().cpu().numpy())
    sim.close()
    return out


def _loss_only(case, prec, nsteps, k, target, bz, v0, v1):
    sim = _sim(case, prec)
    sim.set_driver(_T(bz, prec), _T(v0, prec), _T(v1, prec), case.t0, case.t1)
    sim.set_time(0.0)
    sim.step(nsteps)
    b = sim.bz_plane(sim.read(), k).double().cpu().numpy()
    sim.close()
    return 0.5 * float(((b - target) ** 2).sum())


@pytest.mark.parametrize("prec,tol,eps,k", [(64, 1e-6, 1e-4, 1), (32, 1e-3, 2e-2, 0)])
def test_misfit_gradient_finite_differences(prec, tol, eps, k):
    """B_z misfit on a layer near the photosphere (where the parameters act
    within a few steps) after 8 steps: the gradient from the adjoint
    (DrivenRun + BzPlane autograd functions) against central differences
    along random directions in (B_z, v0, v1)."""
    case = _case(32, 32, 24, seed=4, dt=0.02)
    target = inputs.magnetogram_bipoles(32, 32, 6, seed=99) * 0.5
    nsteps = 8
    loss, gbz, gv0, gv1 = _loss_and_grads(case, prec, nsteps, k, target, slots=2)
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = [rng.standard_normal(case.bz.shape), rng.standard_normal(case.v0.shape) * 0.1,
             rng.standard_normal(case.v1.shape) * 0.1]
        lp = _loss_only(case, prec, nsteps, k, target, case.bz + eps * d[0], case.v0 + eps * d[1], case.v1 + eps * d[2])
        lm = _loss_only(case, prec, nsteps, k, target, case.bz - eps * d[0], case.v0 - eps * d[1], case.v1 - eps * d[2])
        fd = (lp - lm) / (2 * eps)
        ad = float(np.sum(gbz * d[0]) + np.sum(gv0 * d[1]) + np.sum(gv1 * d[2]))
        assert abs(ad) > 1e-6
        assert abs(fd - ad) <= tol * abs(ad), (fd, ad)


@pytest.mark.parametrize("prec", [64, 32])
def test_checkpoint_budget_does_not_change_the_gradient(prec):
    """Binomial checkpointing recomputes the same forward states, and a tape
    keeps exactly the states the recomputation would produce: gradients with
    1 slot, one slot per step, and the whole history taped (27 slots for 9
    steps: three substep states per step, nothing recomputed) are bitwise
    identical."""
    case = _case(16, 16, 12, seed=6)
    target = np.zeros((16, 16))
    a = _loss_and_grads(case, prec, 9, 6, target, slots=1)
    b = _loss_and_grads(case, prec, 9, 6, target, slots=9)
    c = _loss_and_grads(case, prec, 9, 6, target, slots=27)
    assert a[0] == b[0] == c[0]
    for x, y, z in zip(a[1:], b[1:], c[1:]):
        assert np.array_equal(x, y) and np.array_equal(x, z)


@pytest.mark.parametrize("prec", [64, 32])
def test_taped_steps_equal_plain_steps(prec):
    """mhd_step_taped advances the state exactly as mhd_step; its tape holds
    the ghost-filled first state of the step (the state read back after a
    ghost fill); the taped reverse step equals restore + mhd_adjoint_step."""
    case = _case(32, 16, 12, seed=14)
    a, b = _sim(case, prec), _sim(case, prec)
    for sim in (a, b):
        sim.set_driver(_T(case.bz, prec), _T(case.v0, prec), _T(case.v1, prec), case.t0, case.t1)
        sim.set_time(0.0)
    tapes = [b.new_tape() for _ in range(3)]
    a.step(3)
    for tp in tapes:
        b.step_taped(tp)
    assert torch.equal(a.read(), b.read())
    assert a.time() == b.time()
    rng = np.random.default_rng(15)
    lam = _T(rng.standard_normal((8, 12, 16, 32)), prec)
    # reverse of the last step: recompute path from a checkpoint of its
    # first state, against the taped path
    a.set_time(0.0)
    a.write(_T(case.state, prec))
    a.step(2)
    ck = a.new_checkpoint()
    t = a.save(ck)
    a.adjoint_init(lam)
    a.restore(ck, t)
    a.adjoint_step()
    ga = a.adjoint_read()
    b.adjoint_init(lam)
    b.adjoint_step_taped(tapes[2])
    gb = b.adjoint_read()
    for k in ("lam", "bz", "v0", "v1"):
        assert torch.equal(ga[k], gb[k]), k
    a.close()
    b.close()


def test_bruteforce_oracle_gradient_8cube():
    """Every component of the gradient of the B_z misfit on the photosphere
    (8^3 box, 3 steps) against central differences of the FP64 CPU oracle."""
    case = _case(8, 8, 8, seed=8, dt=0.02)
    p = case.params
    k, nsteps = 0, 3
    target = np.sin(np.arange(64).reshape(8, 8) * 0.3) * 0.1
    loss, gbz, gv0, gv1 = _loss_and_grads(case, 64, nsteps, k, target, slots=3)

    def oracle_loss(bz, v0, v1):
        axt, ayt = oracle.a_target(p, bz)
        u = oracle.to_padded(case.state)
        oracle.run(p, u, case.lnrho0, axt, ayt, v0, v1, case.t0, case.t1, 0.0, nsteps)
        oracle.fill_ghosts(p, u, case.lnrho0)
        b = oracle.deriv(p, u, 1, 0, 0)[k] - oracle.deriv(p, u, 0, 0, 1)[k]
        return 0.5 * float(((b - target) ** 2).sum())

    assert abs(oracle_loss(case.bz, case.v0, case.v1) - loss) <= 1e-10 * loss
    eps = 1e-5
    scale = max(np.abs(gbz).max(), np.abs(gv0).max(), np.abs(gv1).max())
    assert scale > 1e-4
    for name, g in (("bz", gbz), ("v0", gv0), ("v1", gv1)):
        base = {"bz": case.bz, "v0": case.v0, "v1": case.v1}
        fd = np.zeros_like(g)
        for idx in np.ndindex(g.shape):
            args_p = {kk: vv.copy() for kk, vv in base.items()}
            args_m = {kk: vv.copy() for kk, vv in base.items()}
            args_p[name][idx] += eps
            args_m[name][idx] -= eps
            fd[idx] = (oracle_loss(args_p["bz"], args_p["v0"], args_p["v1"]) -
                       oracle_loss(args_m["bz"], args_m["v0"], args_m["v1"])) / (2 * eps)
        assert np.abs(fd - g).max() <= 1e-6 * scale, (name, np.abs(fd - g).max(), scale)


def _adjoint_with_variant(case, prec, variant, lam):
    import os
    old = os.environ.get("MHD_ADJ_VARIANT")
    os.environ["MHD_ADJ_VARIANT"] = variant
    try:
        sim = _sim(case, prec)
    finally:
        if old is None:
            del os.environ["MHD_ADJ_VARIANT"]
        else:
            os.environ["MHD_ADJ_VARIANT"] = old
    sim.set_driver(_T(case.bz, prec), _T(case.v0, prec), _T(case.v1, prec), case.t0, case.t1)
    sim.set_time(0.3)
    ck = sim.new_checkpoint()
    t = sim.save(ck)
    sim.adjoint_init(_T(lam, prec))
    sim.restore(ck, t)
    sim.adjoint_step()
    g = sim.adjoint_read()
    out = {k: v.double().cpu().numpy() for k, v in g.items()}
    sim.close()
    return out


@pytest.mark.parametrize("variant", ["tiled", "tiled3d"])
@pytest.mark.parametrize("shape,prec", [((16, 8, 13), 64), ((64, 32, 21), 64), ((64, 32, 21), 32),
                                        ((32, 16, 37), 32), ((128, 32, 21), 32)])
def test_tiled_gather_matches_simple(shape, prec, variant):
    """The shared-memory adjoint kernels ("tiled", the default: the FP32
    pointwise adjoint on the f32x2 / TMEM z-march and a gather that
    z-marches over coefficient planes with a z-scatter register ring;
    "tiled3d": the one-cell-per-thread z-march point kernel and a 3D-tiled
    gather after a grad-div fold) against the one thread per point kernels:
    tiles ragged in x (16 < 32), several y tiles, z chunks ragged (13 + 6,
    21 + 6, 37 + 6 output layers), several tiles in x and y (128 x 32)."""
    nx, ny, nz = shape
    case = _case(nx, ny, nz, seed=12)
    lam = np.random.default_rng(13).standard_normal((8, nz, ny, nx))
    a = _adjoint_with_variant(case, prec, variant, lam)
    b = _adjoint_with_variant(case, prec, "simple", lam)
    tol = 1e-12 if prec == 64 else 1e-5
    for name in ("lam", "bz", "v0", "v1"):
        s = np.abs(b[name]).max()
        assert np.abs(a[name] - b[name]).max() <= tol * max(s, 1e-30), name


def test_gather_with_claimed_work_items_matches_simple():
    """256^3 in FP32: the gather has 2048 work items for the 304 resident CTAs
    of a GB300, so each CTA claims its items from the step state's counter
    (and the point kernel's items run tile-fastest); the result against the
    one thread per point kernels, as in the smaller cases above."""
    case = _case(256, 256, 256, seed=14)
    lam = np.random.default_rng(15).standard_normal((8, 256, 256, 256))
    a = _adjoint_with_variant(case, 32, "tiled", lam)
    b = _adjoint_with_variant(case, 32, "simple", lam)
    for name in ("lam", "bz", "v0", "v1"):
        s = np.abs(b[name]).max()
        assert np.abs(a[name] - b[name]).max() <= 1e-5 * max(s, 1e-30), name
