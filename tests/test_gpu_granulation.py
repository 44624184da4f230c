"""The granulation driver (Sect. 2.3, Eqs. 1-4) through the C ABI against
the oracle (oracle/granulation.py) on the same seeded draws:
- the granule population after each of a run of updates, with births and
  deaths: occupancy bit-exact, parameters to rounding;
- the granular field, the filtered rotational part (Eq. 3) and the output
  (Eq. 4), element by element, FP64 and FP32 outputs;
- edge cases: the smallest plane, a non-square plane, all keys equal
  (ties broken by index: many rounds), an empty plane, f_rot = 0, host
  arrays in and out;
- the 1024 x 1024 plane of the benchmark: the packing invariants
  (independence, fullness, the first key a centre) over the whole plane,
  the granular field at sampled pixels against the oracle's direct sum,
  the rotational part divergence-free and Eq. 4's rms identity.
Tolerances: the GPU and the oracle evaluate the same FP64 formulas in
different orders (and CUDA's exp, log against the host's), so fields agree
to ~1e-15 of their scale; 1e-12 relative to the field's maximum is used
(FP32 output: 2e-7, the float rounding of values up to the maximum)."""
import math

import numpy as np
import pytest

import inputs
from oracle.granulation import GranParams, Granulation as OracleGran

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIX = 0.23  # Mm per pixel, the driver figure's pixel size
GP = dict(r_inner=0.64 / PIX, r_granule=0.8 / PIX, r_lane=1.04 / PIX, v0=1.028, vmin_frac=0.78,
          lifetime=300.0, lifetime_spread=0.10, amp_spread=0.15, f_rot=5.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1908_08557_gb300.build import build
    build()


def _pair(nx, ny, dx, dy, **over):
    from paper_1908_08557_gb300 import Granulation
    gp = dict(GP, **over)
    return Granulation(nx, ny, dx, dy, gp), OracleGran(nx, ny, dx, dy, GranParams(**gp))


def _disk_margin(r, dx, dy):
    """Smallest relative gap between |o|^2 and r^2 over the integer offsets
    near the disk edge (a decision within rounding of the edge could differ
    between two correct evaluations)."""
    m = math.inf
    for oy in range(-int(r / dy) - 2, int(r / dy) + 3):
        for ox in range(-int(r / dx) - 2, int(r / dx) + 3):
            m = min(m, abs((ox * dx) ** 2 + (oy * dy) ** 2 - r * r) / (r * r))
    return m


def _check_population(gen, ref, t):
    occ, par = gen.granules()
    o_occ, o_par = ref.maps()
    assert np.array_equal(occ.cpu().numpy(), o_occ), f"occupancy differs at t={t}"
    np.testing.assert_allclose(par.cpu().numpy(), o_par, rtol=1e-14, atol=0)


def _death_margin(ref, t):
    """Smallest |t - t0 - 2 t_max| / t_max over live granules."""
    return min([abs(t - v[0] - 2 * v[3]) / v[3] for v in ref.live.values()] or [math.inf])


def _close(a, b, tol):
    scale = max(np.max(np.abs(b)), 1e-300)
    assert np.max(np.abs(a - b)) <= tol * scale, np.max(np.abs(a - b)) / scale


@pytest.mark.parametrize("nx,ny,dx,dy", [(64, 64, 1.0, 1.0), (128, 32, 1.0, 1.25), (32, 64, 0.8, 1.0)])
def test_population_and_velocity_over_a_run(nx, ny, dx, dy):
    for r in (GP["r_inner"], GP["r_lane"]):
        assert _disk_margin(r, dx, dy) > 1e-9
    gen, ref = _pair(nx, ny, dx, dy)
    # updates every 40 s over 1.5 lifetimes: births, deaths, refills
    for u, t in enumerate(np.arange(0.0, 480.0, 40.0)):
        assert _death_margin(ref, t) > 1e-9
        draws = inputs.granulation_draws(nx, ny, seed=11, update=u)
        rounds = gen.update(float(t), *draws)
        ref.update(float(t), *draws)
        assert rounds >= 1
        _check_population(gen, ref, t)
        if u % 3 == 2:
            tv = float(t) + 13.0
            v64 = gen.velocity(tv, precision=64).cpu().numpy()
            vg = gen.field(0).cpu().numpy()
            vr = gen.field(1).cpu().numpy()
            ox, oy = ref.granular_field(tv)
            _close(vg, np.stack([ox, oy]), 1e-12)
            from oracle.granulation import rotational_part
            rx, ry = rotational_part(ox, oy, dx, dy)
            _close(vr, np.stack([rx, ry]), 1e-12)
            wx, wy = ref.velocity(tv)
            _close(v64, np.stack([wx, wy]), 1e-12)
            v32 = gen.velocity(tv, precision=32).cpu().numpy()
            _close(v32.astype(np.float64), np.stack([wx, wy]), 2e-7)
    assert len(ref.live) > 0


def test_smallest_plane_and_ties():
    # 8 x 8 plane, lane radius below half the plane; every key equal: the
    # pixels are visited in index order (many rounds)
    over = dict(r_inner=1.6, r_granule=2.0, r_lane=3.5)
    gen, ref = _pair(8, 8, 1.0, 1.0, **over)
    keys = np.full((8, 8), 5, np.uint32)
    _, cl, ca = inputs.granulation_draws(8, 8, seed=3)
    rounds = gen.update(0.0, keys, cl, ca)
    ref.update(0.0, keys, cl, ca)
    _check_population(gen, ref, 0.0)
    assert rounds > 2
    _close(gen.velocity(20.0, precision=64).cpu().numpy(), np.stack(ref.velocity(20.0)), 1e-12)


def test_empty_plane_and_no_rotation():
    gen, ref = _pair(32, 32, 1.0, 1.0, f_rot=0.0)
    v = gen.velocity(0.0, precision=64).cpu().numpy()
    assert np.all(v == 0.0)  # no granules: zero, not NaN
    d = inputs.granulation_draws(32, 32, seed=4)
    gen.update(0.0, *d)
    ref.update(0.0, *d)
    v = gen.velocity(30.0, precision=64).cpu().numpy()
    vg = gen.field(0).cpu().numpy()
    # f_rot = 0: v_vor = v_gran and the Eq. 4 scale is 1 (to rounding)
    _close(v, vg, 1e-14)
    _close(v, np.stack(ref.velocity(30.0)), 1e-12)


def test_host_arrays_in_and_out():
    gen, ref = _pair(64, 32, 1.0, 1.0)
    d = inputs.granulation_draws(64, 32, seed=6)
    gen.update(0.0, *d)                                   # numpy: host path
    ref.update(0.0, *d)
    dev = [torch.as_tensor(a.view(np.int32) if a.dtype == np.uint32 else a, device="cuda") for a in
           inputs.granulation_draws(64, 32, seed=6, update=1)]
    gen.update(200.0, *dev)                               # device path
    ref.update(200.0, *inputs.granulation_draws(64, 32, seed=6, update=1))
    _check_population(gen, ref, 200.0)
    out = np.empty((2, 32, 64), np.float64)
    gen.velocity(230.0, precision=64, out=out)
    _close(out, np.stack(ref.velocity(230.0)), 1e-12)


def test_argument_errors():
    from paper_1908_08557_gb300 import Granulation, MHDError
    with pytest.raises(MHDError):
        Granulation(48, 64, 1.0, 1.0, GP)                 # not a power of two
    with pytest.raises(MHDError):
        Granulation(8, 8, 1.0, 1.0, GP)                   # lane wider than half the plane
    with pytest.raises(MHDError):
        Granulation(64, 64, 1.0, 1.0, dict(GP, vmin_frac=0.9))  # v_min above the lowest v_max


def test_full_plane_invariants():
    n = 1024
    from paper_1908_08557_gb300 import Granulation
    gen = Granulation(n, n, 1.0, 1.0, GP)
    keys, cl, ca = inputs.granulation_draws(n, n, seed=21)
    dk = torch.as_tensor(keys.view(np.int32), device="cuda")
    rounds = gen.update(0.0, dk, torch.as_tensor(cl, device="cuda"), torch.as_tensor(ca, device="cuda"))
    occ, par = gen.granules()
    occ_b = occ.bool()
    # the disk of r_inner, as offsets
    r = GP["r_inner"]
    offs = [(ox, oy) for oy in range(-3, 4) for ox in range(-3, 4) if (ox, oy) != (0, 0) and ox * ox + oy * oy < r * r]
    near = torch.zeros_like(occ_b)
    for ox, oy in offs:
        sh = torch.roll(occ_b, shifts=(oy, ox), dims=(0, 1))
        assert not torch.any(sh & occ_b), "two centres closer than r_inner"
        near |= sh
    assert torch.all(near | occ_b), "a pixel farther than r_inner from every centre"
    q = int(np.lexsort((np.arange(n * n), keys.ravel()))[0])
    assert bool(occ_b.view(-1)[q])
    # parameters at the centres from the draws there
    c = occ_b.cpu().numpy()
    T = par[1].cpu().numpy()[c]
    np.testing.assert_allclose(T, 300.0 * (1 + 0.1 * np.clip(cl[c], -1, 1)), rtol=1e-15)
    # velocity: sampled pixels of v_gran against the oracle's direct sum over
    # the GPU's granules; Eq. 3 divergence-free; Eq. 4 rms identity
    t = 75.0
    v = gen.velocity(t, precision=64)
    vg = gen.field(0)
    ref = OracleGran(n, n, 1.0, 1.0, GranParams(**GP))
    p = par.cpu().numpy()
    for j, i in zip(*np.nonzero(c)):
        ref.live[(int(j), int(i))] = tuple(float(p[m, j, i]) for m in range(4))
    rng = np.random.default_rng(5)
    pix = [tuple(x) for x in rng.integers(0, n, (64, 2))]
    want = ref.granular_field_at(t, pix)
    got = np.array([[vg[0, j, i].item(), vg[1, j, i].item()] for j, i in pix])
    assert np.max(np.abs(got - want)) <= 1e-12 * float(vg.abs().max())
    vr = gen.field(1)
    k = 2 * math.pi * torch.fft.fftfreq(n, device="cuda", dtype=torch.float64)
    div = k[None, :] * torch.fft.fft2(vr[0]) + k[:, None] * torch.fft.fft2(vr[1])
    assert float(div.abs().max()) <= 1e-9 * float(vr.abs().max()) * n
    assert float((v ** 2).sum()) == pytest.approx(float((vg ** 2).sum()), rel=1e-12)
    assert rounds < 200
    assert gen.launch_count() > 0
