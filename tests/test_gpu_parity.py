"""GPU parity: every kernel of libmhd, called through the C ABI, against the
FP64 CPU oracle on the same seeded inputs.

Tolerances: the FP64 path agrees with the oracle to rounding (1e-11 relative
L2 per field after 50 steps); the FP32 path to 1e-4 per field after 50 steps
(FP32 state and stencils, FP64 FFT and reductions).
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


def _sim(case, precision, stats_every=0, driver=True, params=None, lnT0=True):
    from paper_1908_08557_gb300 import Simulation
    p = params or case.params
    dt = torch.float64 if precision == 64 else torch.float32
    sim = Simulation(p, torch.tensor(case.state, dtype=dt, device="cuda"), case.lnrho0,
                     case.lnT0 if lnT0 else None, precision=precision, stats_every=stats_every)
    if driver:
        sim.set_driver(torch.tensor(case.bz, dtype=dt, device="cuda"),
                       torch.tensor(case.v0, dtype=dt, device="cuda"),
                       torch.tensor(case.v1, dtype=dt, device="cuda"), case.t0, case.t1)
    return sim


def _perturbed(nx, ny, nz, seed, **kw):
    case = inputs.make_box(nx, ny, nz, seed=seed, **kw)
    rng = np.random.default_rng(seed + 100)
    st = case.state.copy()
    st[3:6] += 0.05 * rng.standard_normal(st[3:6].shape)
    st[7] += 0.02 * rng.standard_normal(st[7].shape)
    st[0:3] += 0.01 * rng.standard_normal(st[0:3].shape)
    case.state = st
    return case


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("shape", [(16, 16, 12), (32, 8, 9), (8, 64, 7)])
def test_ghost_fill_fp64(shape):
    nx, ny, nz = shape
    case = _perturbed(nx, ny, nz, seed=1)
    sim = _sim(case, 64)
    sim.fill_ghosts()
    got = sim.read_padded(0)
    u = oracle.to_padded(case.state)
    oracle.fill_ghosts(case.params, u, case.lnrho0)
    scale = np.abs(u).max(axis=(1, 2, 3))
    err = np.abs(got - u).max(axis=(1, 2, 3))
    assert np.all(err <= 1e-13 * scale), err / scale


def test_ghost_fill_periodic_z_ragged():
    case = _perturbed(40, 24, 20, seed=2)
    p = dict(case.params, bc_z=1)
    sim = _sim(case, 64, driver=False, params=p)
    sim.fill_ghosts()
    got = sim.read_padded(0)
    u = oracle.to_padded(case.state)
    oracle.fill_ghosts(p, u, case.lnrho0)
    assert np.array_equal(got[:, :, :, :], u)


def test_magnetogram_inversion_fp64():
    case = inputs.make_box(32, 16, 8, seed=4, dy=1.5)
    sim = _sim(case, 64)
    ax, ay = oracle.a_target(case.params, case.bz)
    got = sim.read_target()
    s = np.abs(np.stack([ax, ay])).max()
    assert np.abs(got[0] - ax).max() < 1e-13 * s
    assert np.abs(got[1] - ay).max() < 1e-13 * s


@pytest.mark.parametrize("shape,bcz", [((16, 16, 12), 0), ((32, 16, 10), 0), ((40, 24, 20), 1)])
def test_rhs_fp64(shape, bcz):
    nx, ny, nz = shape
    case = _perturbed(nx, ny, nz, seed=3)
    p = dict(case.params, bc_z=bcz)
    sim = _sim(case, 64, params=p, driver=(bcz == 0))
    sim.fill_ghosts()
    t = 0.37
    got = sim.eval_rhs(t)
    u = sim.read_padded(0).astype(np.float64)
    if bcz == 0:
        axt, ayt = oracle.a_target(p, case.bz)
        v0, v1 = case.v0, case.v1
    else:
        axt = ayt = np.zeros((ny, nx))
        v0 = v1 = np.zeros((2, ny, nx))
    ref = oracle.rhs(p, u, axt, ayt, v0, v1, case.t0, case.t1, t)
    for f in range(8):
        s = np.abs(ref[f]).max()
        e = np.abs(got[f] - ref[f]).max()
        assert e <= 1e-11 * max(s, 1e-30), (f, e, s)


def test_rhs_fp32():
    case = _perturbed(16, 16, 12, seed=5)
    sim = _sim(case, 32)
    sim.fill_ghosts()
    got = sim.eval_rhs(0.2).astype(np.float64)
    u = sim.read_padded(0).astype(np.float64)
    axt, ayt = (a.astype(np.float32).astype(np.float64) for a in oracle.a_target(case.params, case.bz))
    ref = oracle.rhs(case.params, u, axt, ayt, case.v0.astype(np.float32).astype(np.float64),
                     case.v1.astype(np.float32).astype(np.float64), case.t0, case.t1, 0.2)
    for f in range(8):
        s = np.abs(ref[f]).max()
        e = np.abs(got[f] - ref[f]).max()
        assert e <= 2e-4 * max(s, 1e-30), (f, e, s)


def test_cfl_and_stats_fp64():
    case = _perturbed(32, 32, 16, seed=6)
    sim = _sim(case, 64)
    sim.fill_ghosts()
    u = sim.read_padded(0)
    dt = sim.compute_dt()
    assert abs(dt - oracle.cfl(case.params, u)) <= 1e-13 * dt
    st = sim.compute_stats()
    ref = oracle.stats(case.params, u)
    keys = ["e_kin", "e_mag", "e_th", "mass", "flux_net", "flux_abs", "divb_max"]
    for q, k in enumerate(keys[:4] + keys[5:6]):
        r = ref[keys.index(k)]
        assert abs(st[k] - r) <= 1e-12 * abs(r), (k, st[k], r)
    assert abs(st["flux_net"] - ref[4]) <= 1e-12 * ref[5]
    assert st["divb_max"] < 1e-10 and ref[6] < 1e-10


@pytest.mark.parametrize("shape,precision", [((16, 8, 11), 64), ((64, 32, 21), 32), ((16, 8, 11), 32)])
def test_stats_ragged_and_in_step(shape, precision):
    """Diagnostics on tiles with ragged x, y and z extents, in both precisions,
    against the oracle; the in-step diagnostics (taken at the start of a step,
    with B staged in the RK accumulator) equal the standalone call bit for bit,
    and leave the step itself unchanged."""
    case = _perturbed(*shape, seed=11)
    sim = _sim(case, precision, stats_every=1)
    sim.fill_ghosts()
    u = sim.read_padded(0)
    st = sim.compute_stats()
    ref = oracle.stats(case.params, np.ascontiguousarray(u, dtype=np.float64))
    keys = ["e_kin", "e_mag", "e_th", "mass", "flux_net", "flux_abs", "divb_max"]
    tol = 1e-12 if precision == 64 else 1e-5
    for k in ("e_kin", "e_mag", "e_th", "mass", "flux_abs"):
        r = ref[keys.index(k)]
        assert abs(st[k] - r) <= tol * abs(r), (k, st[k], r)
    assert abs(st["flux_net"] - ref[4]) <= tol * ref[5]
    # |div B| relative to |B| / dx: rounding of the curl and divergence stencils
    dx = case.params["dx"]
    bscale = np.sqrt(2.0 * ref[1] / (shape[0] * shape[1] * shape[2] * dx ** 3)) / dx
    assert st["divb_max"] <= (1e-10 if precision == 64 else 1e-3) * bscale, (st["divb_max"], bscale)
    sim.step(1)
    st2 = sim.read_stats()
    for k in keys:
        assert st2[k] == st[k], (k, st2[k], st[k])
    ref_sim = _sim(case, precision, stats_every=0)
    ref_sim.step(1)
    assert torch.equal(sim.read(), ref_sim.read())


def test_full_run_fp64_spots4_32():
    """Workload spots4_32x32x32 (4 spots, 50 RK3 steps): FP64 GPU vs oracle,
    relative L2 <= 1e-11 per field, same time."""
    case = inputs.make_case("spots4_32x32x32")
    sim = _sim(case, 64)
    sim.step(case.nsteps)
    got = sim.read().cpu().numpy()
    u, t, dts = oracle.run_case(case)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    assert max(errs) <= 1e-11, errs
    tg, dtg = sim.time()
    assert abs(tg - t) <= 1e-12 * t
    # stateful horizontal-velocity ghosts below the photosphere
    gp = sim.read_padded(0)
    for c in (3, 4):
        a = gp[c, :NG, NG:-NG, NG:-NG]
        b = u[c, :NG, NG:-NG, NG:-NG]
        assert _rel_l2(a, b) <= 1e-11


def test_full_run_fp32_spots4_32():
    """Same workload on the FP32 path: relative L2 <= 1e-4 per field."""
    case = inputs.make_case("spots4_32x32x32")
    sim = _sim(case, 32)
    sim.step(case.nsteps)
    got = sim.read().cpu().numpy().astype(np.float64)
    u, t, dts = oracle.run_case(case)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    print("fp32 rel L2 per field:", ["%.2e" % e for e in errs])
    assert max(errs) <= 1e-4, errs


def test_periodic_ragged_run_fp64():
    case = _perturbed(40, 24, 20, seed=7)
    p = dict(case.params, bc_z=1, eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0, gz=0.0)
    sim = _sim(case, 64, params=p, driver=False)
    sim.step(5)
    got = sim.read().cpu().numpy()
    z2 = np.zeros((24, 40)); v2 = np.zeros((2, 24, 40))
    u = oracle.to_padded(case.state)
    oracle.run(p, u, case.lnrho0, z2, z2, v2, v2, 0.0, 1.0, 0.0, 5)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    assert max(errs) <= 1e-12, errs


@pytest.mark.parametrize("precision", [64, 32])
def test_periodic_odd_nx_cfl_and_stats(precision):
    """Odd nx in the periodic test geometry: the CFL and diagnostics kernels
    work on x pairs, the last of which has one cell outside the box."""
    case = _perturbed(37, 22, 13, seed=9)
    p = dict(case.params, bc_z=1, eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0, gz=0.0)
    sim = _sim(case, precision, params=p, driver=False)
    sim.fill_ghosts()
    u = np.ascontiguousarray(sim.read_padded(0), dtype=np.float64)
    tol = 1e-12 if precision == 64 else 1e-5
    dt = sim.compute_dt()
    assert abs(dt - oracle.cfl(p, u)) <= tol * dt
    st = sim.compute_stats()
    ref = oracle.stats(p, u)
    keys = ["e_kin", "e_mag", "e_th", "mass", "flux_net", "flux_abs", "divb_max"]
    for k in ("e_kin", "e_mag", "e_th", "mass", "flux_abs"):
        r = ref[keys.index(k)]
        assert abs(st[k] - r) <= tol * abs(r), (k, st[k], r)
    assert abs(st["flux_net"] - ref[4]) <= tol * ref[5]
    bscale = np.sqrt(2.0 * ref[1] / (37 * 22 * 13 * p["dx"] ** 3)) / p["dx"]
    assert st["divb_max"] <= (1e-10 if precision == 64 else 1e-3) * bscale


@pytest.mark.parametrize("precision", [64, 32])
def test_minimum_size_run(precision):
    """The smallest box the FFT boundary and the pair kernel take (8 x 8
    horizontal points, 7 layers): step(0) changes nothing; 5 steps against
    the oracle."""
    case = _perturbed(8, 8, 7, seed=12)
    sim = _sim(case, precision)
    before = sim.read().clone()
    sim.step(0)
    assert torch.equal(sim.read(), before) and sim.time()[0] == 0.0
    sim.step(5)
    got = sim.read().cpu().numpy().astype(np.float64)
    u, t, dts = oracle.run_case(case, nsteps=5)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    assert max(errs) <= (1e-11 if precision == 64 else 1e-4), errs
    assert abs(sim.time()[0] - t) <= (1e-12 if precision == 64 else 1e-5) * t


NC = dict(nc_tau=0.5, nc_z_max=10.0, nc_z_width=3.0)


def _cooling_case(nx, ny, nz, seed):
    """A perturbed box with Newtonian cooling on (Sect. 3.1); ln rho is
    perturbed too, so the local densities fall between the layers' initial
    values and the inverse lookup interpolates."""
    case = _perturbed(nx, ny, nz, seed=seed)
    rng = np.random.default_rng(seed + 300)
    case.state[6] += 0.05 * rng.standard_normal(case.state[6].shape)
    case.params = dict(case.params, **NC)
    oracle.set_nc_profile(case.lnrho0, case.lnT0)
    return case


@pytest.mark.parametrize("variant", ["fp64", "pair", "tiled", "fused", "simple"])
def test_cooling_rhs(variant):
    """Right-hand side with Newtonian cooling against the oracle: the FP64
    kernel to 1e-11 of each field's scale, each FP32 kernel to 2e-4."""
    case = _cooling_case(16, 16, 16, seed=21)
    p = case.params
    t = 0.31
    if variant == "fp64":
        sim = _sim(case, 64)
        sim.fill_ghosts()
        got = sim.eval_rhs(t)
        u = sim.read_padded(0).astype(np.float64)
        sim.close()
        axt, ayt = oracle.a_target(p, case.bz)
        v0, v1, tol = case.v0, case.v1, 1e-11
    else:
        got, u = _eval_with_variant(case, variant, t=t)
        cast = lambda a: a.astype(np.float32).astype(np.float64)
        axt, ayt = (cast(a) for a in oracle.a_target(p, case.bz))
        v0, v1, tol = cast(case.v0), cast(case.v1), 2e-4
    ref = oracle.rhs(p, u, axt, ayt, v0, v1, case.t0, case.t1, t)
    for f in range(8):
        s = np.abs(ref[f]).max()
        e = np.abs(got[f] - ref[f]).max()
        assert e <= tol * max(s, 1e-30), (f, e, s)
    # the term is active: the same state without it differs in ln T only
    off = oracle.rhs(dict(p, nc_tau=0.0), u, axt, ayt, v0, v1, case.t0, case.t1, t)
    assert np.abs(off[7] - ref[7]).max() > 1e-4
    assert all(np.array_equal(off[f], ref[f]) for f in range(7))


@pytest.mark.parametrize("precision,tol", [(64, 1e-11), (32, 1e-4)])
def test_cooling_full_run(precision, tol):
    """Workload spots4_32x32x32 with Newtonian cooling on (rate 0.5, height
    cut-off over layers 7-10): 50 steps against the oracle."""
    case = inputs.make_case("spots4_32x32x32")
    p = dict(case.params, **NC)
    oracle.set_nc_profile(case.lnrho0, case.lnT0)
    sim = _sim(case, precision, params=p)
    sim.step(case.nsteps)
    got = sim.read().cpu().numpy().astype(np.float64)
    u, t, dts = oracle.run_case(case, params=p)
    ref = oracle.interior(u)
    errs = [_rel_l2(got[f], ref[f]) for f in range(8)]
    assert max(errs) <= tol, errs


def test_steps_captured_in_a_cuda_graph():
    """Two RK steps captured in a CUDA graph on the handle's stream (the
    substep-0 FFT forks to the side stream and joins back inside the capture)
    and replayed twice equal four eagerly launched steps bit for bit: the
    time step, substep times and driver weights live on the device, and two
    steps (six substeps) return the ping-pong state sets to where they were."""
    from paper_1908_08557_gb300 import Simulation
    case = inputs.make_case("spots4_32x32x32")
    s = torch.cuda.Stream()

    def make(stream):
        sim = Simulation(case.params, torch.tensor(case.state, dtype=torch.float32, device="cuda"), case.lnrho0,
                         case.lnT0, precision=32, stream=stream)
        sim.set_driver(torch.tensor(case.bz, dtype=torch.float32, device="cuda"),
                       torch.tensor(case.v0, dtype=torch.float32, device="cuda"),
                       torch.tensor(case.v1, dtype=torch.float32, device="cuda"), case.t0, case.t1)
        return sim

    sg, se = make(s), make(None)
    with torch.cuda.stream(s):
        sg.step(2)  # first launches (one-time kernel attributes) outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sg.step(2)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    se.step(6)
    torch.cuda.synchronize()
    assert torch.equal(sg.read(), se.read())
    assert sg.time()[0] == se.time()[0]


def test_nonfinite_detected():
    from paper_1908_08557_gb300 import MHDError
    from paper_1908_08557_gb300.binding import MHD_ERR_NONFINITE
    case = inputs.make_box(16, 16, 10, seed=8)
    st = case.state.copy()
    st[7, 4, 5, 6] = np.nan
    case.state = st
    sim = _sim(case, 32)
    sim.step(2)
    with pytest.raises(MHDError) as e:
        sim.time()
    assert e.value.code == MHD_ERR_NONFINITE


def _eval_with_variant(case, variant, t=0.29, params=None, driver=True):
    import os
    old = os.environ.get("MHD_RK_VARIANT")
    os.environ["MHD_RK_VARIANT"] = variant
    try:
        sim = _sim(case, 32, params=params, driver=driver)
    finally:
        if old is None:
            del os.environ["MHD_RK_VARIANT"]
        else:
            os.environ["MHD_RK_VARIANT"] = old
    sim.fill_ghosts()
    out = sim.eval_rhs(t).astype(np.float64)
    u = sim.read_padded(0).astype(np.float64)
    sim.close()
    return out, u


@pytest.mark.parametrize("variant", ["pair", "tiled", "fused"])
@pytest.mark.parametrize("shape,bcz", [((16, 16, 12), 0), ((64, 32, 41), 0), ((40, 24, 20), 1)])
def test_tiled_kernel_matches_simple_fp32(shape, bcz, variant):
    """The TMA-fed z-march kernels (default "pair": one pass, two cells per
    thread in f32x2, z histories in TMEM; "tiled": the split A / rest
    passes; "fused": one pass over all 8 fields, one cell per thread)
    against the one-thread-per-cell kernel: same FP32 discretisation,
    different summation order; tiles ragged in x (16 < 32) and chunks
    ragged in z (41 layers)."""
    nx, ny, nz = shape
    case = _perturbed(nx, ny, nz, seed=11)
    p = dict(case.params, bc_z=bcz)
    a, ua = _eval_with_variant(case, variant, params=p, driver=(bcz == 0))
    b, ub = _eval_with_variant(case, "simple", params=p, driver=(bcz == 0))
    assert np.array_equal(ua, ub)
    for f in range(8):
        s = np.abs(b[f]).max()
        assert np.abs(a[f] - b[f]).max() <= 2e-5 * max(s, 1e-30), f


def test_pair_kernel_with_claimed_work_items():
    """A launch with a dozen or more work items per CTA (1024 x 1024 x 16:
    4096 tiles of one z chunk each on 304 CTAs) claims its items from a
    counter instead of taking them by grid stride; the right-hand side
    equals the one-thread-per-cell kernel's to the same tolerance."""
    case = _perturbed(1024, 1024, 16, seed=12, magnetogram="bipoles", n_mag=40)
    a, ua = _eval_with_variant(case, "pair")
    b, ub = _eval_with_variant(case, "simple")
    assert np.array_equal(ua, ub)
    for f in range(8):
        s = np.abs(b[f]).max()
        assert np.abs(a[f] - b[f]).max() <= 2e-5 * max(s, 1e-30), f


def test_tiled_full_size_sampled_bipoles40_256():
    """Bench workload bipoles40_256x256x256 in the bench configuration (FP32,
    the default z-march kernel rk_pair_kernel): ghost fill + RHS at 3000 sampled cells -- random, plus the
    photosphere, the top layer, the swamp and the x,y edges -- against the
    FP64 oracle, which fills its own ghosts (plain DFT) and evaluates the
    sampled cells one by one.  Both sides start from the same values: A and u
    rounded to FP32, ln rho and ln T the exact FP64 profiles (the GPU stores
    them as zero perturbations about those profiles)."""
    case = inputs.make_case("bipoles40_256x256x256")
    rng = np.random.default_rng(0)
    st = case.state.copy()
    st[3:6] += 0.01 * rng.standard_normal(st[3:6].shape)
    st[0:6] = st[0:6].astype(np.float32).astype(np.float64)
    case.state = st
    sim = _sim(case, 32)
    sim.fill_ghosts()
    t = 0.21
    got = sim.eval_rhs(t)
    sim.close()
    p = case.params
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    u = oracle.to_padded(st)
    oracle.fill_ghosts(p, u, case.lnrho0)
    ks = np.concatenate([rng.integers(0, nz, 2000), np.zeros(300, int), np.full(300, nz - 1),
                         rng.integers(nz - 5, nz, 200), rng.integers(0, nz, 200)])
    js = rng.integers(0, ny, len(ks))
    iss = rng.integers(0, nx, len(ks))
    iss[-200:] = rng.choice([0, 1, 2, nx - 3, nx - 2, nx - 1], 200)
    js[-100:] = rng.choice([0, 1, 2, ny - 3, ny - 2, ny - 1], 100)
    cells = np.stack([ks, js, iss], axis=1)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    axt, ayt = (f32(x) for x in oracle.a_target(p, case.bz))
    ref = oracle.rhs_cells(p, u, axt, ayt, f32(case.v0), f32(case.v1), case.t0, case.t1, t, cells)
    g = got[:, ks + NG, js + NG, iss + NG].T.astype(np.float64)
    for f in range(8):
        s = np.abs(ref[:, f]).max()
        assert np.abs(g[:, f] - ref[:, f]).max() <= 2e-4 * max(s, 1e-30), (f, np.abs(g[:, f] - ref[:, f]).max(), s)


@pytest.mark.parametrize("prec", [64, 32])
def test_production_geometry_1024_sampled(prec):
    """Production geometry: 1024 x 1024 horizontal points, horizontal spacing
    4x vertical (workload ar_1024x1024x256 recipe on 8 layers): the full
    ghost fill (1024^2 FFT planes; FP64) and the RHS at 3000 sampled cells
    against the oracle (potential-field ghosts by numpy's FFT).  |A| reaches
    several hundred here; the FP32 handle stores A about the FP64 initial
    field (a_background), so its rounding scales with the perturbation and
    the plain FP32 tolerance applies (1e-4 of each row's sampled scale)."""
    case = inputs.make_box(1024, 1024, 8, seed=3, dx=4.0, dy=4.0, magnetogram="bipoles", n_mag=400,
                           driver="solenoidal", ar_pair=(5.0, 40.0, 200.0))
    rng = np.random.default_rng(1)
    st = case.state.copy()
    a0 = st[0:3].copy()
    assert np.abs(a0).max() > 100.0
    st[3:6] += 0.01 * rng.standard_normal(st[3:6].shape)
    if prec == 32:
        st[3:8] = st[3:8].astype(np.float32).astype(np.float64)
    case.state = st
    if prec == 64:
        sim = _sim(case, prec)
    else:
        from paper_1908_08557_gb300 import Simulation
        f32 = dict(dtype=torch.float32, device="cuda")
        sim = Simulation(case.params, torch.tensor(st, **f32), case.lnrho0, case.lnT0, precision=32,
                         a_background=a0)
        sim.set_driver(torch.tensor(case.bz, **f32), torch.tensor(case.v0, **f32), torch.tensor(case.v1, **f32),
                       case.t0, case.t1)
    sim.fill_ghosts()
    p = case.params
    u = oracle.to_padded(st)
    oracle.fill_ghosts(p, u, case.lnrho0, pfe="fft")
    if prec == 64:
        got = sim.read_padded(0)
        for f in range(8):
            scale = np.abs(u[f]).max()
            assert np.abs(got[f] - u[f]).max() <= 1e-12 * scale, f
        del got
    t = 0.4
    rhs = sim.eval_rhs(t)
    sim.close()
    nx, ny, nz = 1024, 1024, 8
    ks = rng.integers(0, nz, 3000)
    js = rng.integers(0, ny, 3000)
    iss = rng.integers(0, nx, 3000)
    cells = np.stack([ks, js, iss], axis=1)
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if prec == 32 else (lambda a: a)
    # the FP32 handle forms its nudging target difference in FP64 from its
    # FP32 copy of B_z
    axt, ayt = oracle.a_target_fft(p, cast(case.bz))
    ref = oracle.rhs_cells(p, u, axt, ayt, cast(case.v0), cast(case.v1), case.t0, case.t1, t, cells)
    g = rhs[:, ks + NG, js + NG, iss + NG].T.astype(np.float64)
    tol = 1e-10 if prec == 64 else 1e-4
    for f in range(8):
        s = np.abs(ref[:, f]).max()
        err = np.abs(g[:, f] - ref[:, f])
        worst = int(np.argmax(err))
        assert err[worst] <= tol * max(s, 1e-30), (f, err[worst], s)


@pytest.mark.parametrize("variant", ["plain", "ragged", "background", "zgrid", "thin7", "thin8"])
def test_in_step_cfl_equals_standalone_fp32(variant):
    """The step's CFL reduction on the FP32 state (the TMA-fed z-march over
    the inner layers, the plane-parallel kernel over the three layers at each
    end) gives the time step of the standalone plane-parallel reduction over
    all layers bit for bit: same arithmetic per cell, order-independent
    maxima.  A tile ragged in x (nx = 16) and ragged z chunks; A about a
    background (its B added per cell); a stretched grid (metric per layer)."""
    from paper_1908_08557_gb300 import Simulation
    kw = {}
    if variant == "zgrid":
        z, _, _ = inputs.stretched_z(40, 0.5, 1.5, 20, 4)
        case = _perturbed(32, 16, 40, seed=81, z=z, magnetogram="bipoles", n_mag=6)
    elif variant == "ragged":
        case = _perturbed(16, 16, 37, seed=82, magnetogram="bipoles", n_mag=6)
    elif variant.startswith("thin"):
        # the thinnest boxes (nz >= 7): one and two inner layers
        case = _perturbed(32, 16, int(variant[4:]), seed=84, magnetogram="bipoles", n_mag=6)
    else:
        case = _perturbed(64, 32, 41, seed=83, magnetogram="bipoles", n_mag=6)
    if variant == "background":
        kw["a_background"] = case.state[0:3] - 0.003
    T = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    sim = Simulation(case.params, T(case.state), case.lnrho0, case.lnT0, precision=32, **kw)
    if variant == "background":
        sim.set_a_background(kw["a_background"], T(np.full(case.state[0:3].shape, 0.003)))
    sim.set_driver(T(case.bz), T(case.v0), T(case.v1), case.t0, case.t1)
    for _ in range(3):
        sim.fill_ghosts()
        dt0 = sim.compute_dt()
        t0 = sim.time()[0]
        sim.step(1)
        t1, dt1 = sim.time()
        assert dt1 == dt0 and t1 == t0 + dt0, (dt0, dt1)
    sim.close()
