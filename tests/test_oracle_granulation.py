"""Pins of the granulation-driver oracle (oracle/granulation.py; Sect. 2.3,
Eqs. 1-4) against what the section and the mathematics fix:
- Eqs. 1-2: a granule is born at v_min, peaks at v_max at t0 + t_max and is
  back at v_min at t0 + 2 t_max, where it is removed;
- placement: centres at least r_inner apart, the plane full (every pixel
  within r_inner of a centre), the first key always a centre, live granules
  blocking their disks, and the lattice that raster order gives in closed
  form;
- the radial field of one granule at known distances, and superposition;
- Eq. 3: the rotational part of a band-limited gradient field vanishes, a
  band-limited solenoidal mode passes times exp(-(2|k|/k_N)^4), and the
  result of any field is divergence-free with zero mean;
- Eq. 4: the output's rms speed equals the granular field's.
"""
import math

import numpy as np
import pytest

from oracle.granulation import (GranParams, Granulation, amplitude, radial_profile, renormalise,
                                rotational_part, t_max)


def _draws(nx, ny, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 32, (ny, nx), dtype=np.uint64).astype(np.uint32)
    return keys, rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))


GP = GranParams(r_inner=2.8, r_granule=3.5, r_lane=4.5, v0=1.0, lifetime=300.0)


@pytest.mark.parametrize("vmax_frac", [0.85, 1.0, 1.15])
def test_life_cycle_closed_forms(vmax_frac):
    T, vmin = 290.0, 0.78
    vm = vmax_frac
    tm = t_max(T, vm, vmin)
    t0 = 17.0
    assert amplitude(t0, t0, T, vm, tm) == pytest.approx(vmin, rel=1e-14)
    assert amplitude(t0 + tm, t0, T, vm, tm) == vm
    assert amplitude(t0 + 2 * tm, t0, T, vm, tm) == pytest.approx(vmin, rel=1e-14)
    # rises before the peak, falls after it
    assert amplitude(t0 + 0.5 * tm, t0, T, vm, tm) > vmin
    assert amplitude(t0 + 2.5 * tm, t0, T, vm, tm) < vmin


def test_expiry_at_twice_the_peak_time():
    g = Granulation(16, 16, 1.0, 1.0, GP)
    k, a, b = _draws(16, 16, 0)
    g.place(0.0, k, a, b)
    (t0, T, vm, tm) = next(iter(g.live.values()))
    n = len(g.live)
    g.expire(0.999 * 2 * tm)
    assert len(g.live) > 0
    longest = max(v[3] for v in g.live.values())
    g.expire(2 * longest * 1.001)
    assert len(g.live) == 0 and n > 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_placement_is_a_full_packing(seed):
    nx, ny = 40, 24
    g = Granulation(nx, ny, 1.0, 1.25, GP)
    keys, a, b = _draws(nx, ny, seed)
    g.place(0.0, keys, a, b)
    c = np.array(list(g.live.keys()))
    r2 = GP.r_inner ** 2
    # independent: no two centres closer than r_inner
    for j, i in c:
        d = g._dist2(j, i, c[:, 0], c[:, 1])
        assert np.sum(d < r2) == 1  # itself only
    # full: every pixel is within r_inner of a centre
    for j in range(ny):
        for i in range(nx):
            assert np.min(g._dist2(j, i, c[:, 0], c[:, 1])) < r2
    # the first pixel visited always starts a granule
    q = int(np.lexsort((np.arange(nx * ny), keys.ravel()))[0])
    assert divmod(q, nx) in g.live
    # parameters from the draws at the centre, clipped to [-1, 1]
    for (j, i), (t0, T, vm, tm) in g.live.items():
        cl = max(-1.0, min(1.0, a[j, i]))
        assert T == GP.lifetime * (1 + 0.1 * cl) and t0 == 0.0
        assert 0.85 * GP.v0 <= vm <= 1.15 * GP.v0


@pytest.mark.parametrize("r_inner", [1.5, 2.0])
def test_raster_order_lattice(r_inner):
    # keys all equal: pixels visited in index order; with r_inner 1.5 or 2 on
    # a unit grid (a centre exactly r_inner away is allowed) the accepted
    # centres are every other pixel of every other row
    gp = GranParams(r_inner=r_inner, r_granule=1.0, r_lane=2.0)
    g = Granulation(16, 16, 1.0, 1.0, gp)
    z = np.zeros((16, 16))
    g.place(0.0, np.zeros((16, 16), np.uint32), z, z)
    assert set(g.live) == {(j, i) for j in range(0, 16, 2) for i in range(0, 16, 2)}


def test_live_granules_block_their_disk():
    g = Granulation(32, 32, 1.0, 1.0, GP)
    g.live[(10, 20)] = (-50.0, 300.0, 1.0, 100.0)
    keys, a, b = _draws(32, 32, 5)
    g.place(0.0, keys, a, b)
    assert g.live[(10, 20)] == (-50.0, 300.0, 1.0, 100.0)
    for (j, i) in g.live:
        if (j, i) != (10, 20):
            assert g._dist2(j, i, 10, 20) >= GP.r_inner ** 2


def test_single_granule_field():
    nx = ny = 32
    g = Granulation(nx, ny, 1.0, 1.0, GP)
    g.live[(5, 30)] = (0.0, 300.0, 1.1, 80.0)
    t = 30.0
    a = 1.1 * math.exp(-((t - 80.0) / 300.0) ** 2)
    vx, vy = g.granular_field(t)
    # (3 px right of the centre, wrapping in x): rise region r / r_g
    assert vx[5, 1] == pytest.approx(a * 3.0 / 3.5, rel=1e-14) and vy[5, 1] == 0.0
    # 4 px below: fall region, cos^2(pi/2 (4 - 3.5) / 1) = 1/2
    assert vy[1, 30] == pytest.approx(-a * 0.5, rel=1e-14) and abs(vx[1, 30]) < 1e-17
    # diagonal (3, 3): r = 3 sqrt 2 = 4.243 in the lane
    r = 3 * math.sqrt(2)
    f = a * math.cos(0.5 * math.pi * (r - 3.5)) ** 2 / math.sqrt(2)
    assert vx[8, 1] == pytest.approx(f, rel=1e-13) and vy[8, 1] == pytest.approx(f, rel=1e-13)
    # the centre and everything from r_lane on are still
    assert vx[5, 30] == 0.0 and vy[5, 30] == 0.0
    far = np.hypot(((np.arange(nx) - 30 + 16) % 32 - 16)[None, :], ((np.arange(ny) - 5 + 16) % 32 - 16)[:, None])
    assert np.all(vx[far >= 4.5] == 0.0) and np.all(vy[far >= 4.5] == 0.0)


def test_profile_values():
    r = np.array([0.0, 1.75, 3.5, 4.0, 4.5, 9.0])
    assert np.allclose(radial_profile(r, 3.5, 4.5), [0.0, 0.5, 1.0, 0.5, 0.0, 0.0], atol=1e-15)


def test_superposition():
    g1 = Granulation(24, 24, 1.0, 1.0, GP)
    g2 = Granulation(24, 24, 1.0, 1.0, GP)
    g12 = Granulation(24, 24, 1.0, 1.0, GP)
    a, b = (3, 4), (6, 7)
    g1.live[a] = g12.live[a] = (0.0, 300.0, 1.0, 90.0)
    g2.live[b] = g12.live[b] = (10.0, 280.0, 0.9, 85.0)
    v1, v2, v12 = g1.granular_field(40.0), g2.granular_field(40.0), g12.granular_field(40.0)
    assert np.allclose(v12[0], v1[0] + v2[0], rtol=0, atol=1e-15)
    assert np.allclose(v12[1], v1[1] + v2[1], rtol=0, atol=1e-15)


def _grid(nx, ny, dx, dy):
    x = (np.arange(nx) * dx)[None, :]
    y = (np.arange(ny) * dy)[:, None]
    return np.broadcast_arrays(x, y)


def test_rotational_part_of_a_gradient_vanishes():
    nx, ny, dx, dy = 32, 16, 1.0, 1.5
    x, y = _grid(nx, ny, dx, dy)
    ax, ay = 2 * np.pi / (nx * dx), 2 * np.pi / (ny * dy)
    # phi = cos(3 ax x) sin(2 ay y) + sin(ax x): grad phi
    vx = -3 * ax * np.sin(3 * ax * x) * np.sin(2 * ay * y) + ax * np.cos(ax * x)
    vy = 2 * ay * np.cos(3 * ax * x) * np.cos(2 * ay * y)
    rx, ry = rotational_part(vx, vy, dx, dy)
    assert np.max(np.abs(rx)) < 1e-14 and np.max(np.abs(ry)) < 1e-14


@pytest.mark.parametrize("m,n", [(1, 0), (3, 2), (5, -4), (0, 3)])
def test_solenoidal_mode_passes_filtered(m, n):
    nx, ny, dx, dy = 32, 16, 1.0, 1.5
    x, y = _grid(nx, ny, dx, dy)
    kx, ky = 2 * np.pi * m / (nx * dx), 2 * np.pi * n / (ny * dy)
    # psi = sin(kx x + ky y): v = (d psi / dy, -d psi / dx)
    c = np.cos(kx * x + ky * y)
    vx, vy = ky * c, -kx * c
    rx, ry = rotational_part(vx, vy, dx, dy)
    kn = math.hypot(kx * dx / math.pi, ky * dy / math.pi)
    w = math.exp(-(2 * kn) ** 4)
    assert np.allclose(rx, w * vx, rtol=0, atol=1e-14) and np.allclose(ry, w * vy, rtol=0, atol=1e-14)


def test_rotational_part_is_divergence_free():
    rng = np.random.default_rng(3)
    vx, vy = rng.standard_normal((2, 16, 32))
    rx, ry = rotational_part(vx, vy, 1.0, 1.0)
    kx = 2 * np.pi * np.fft.fftfreq(32)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(16)[:, None]
    div = kx * np.fft.fft2(rx) + ky * np.fft.fft2(ry)
    assert np.max(np.abs(div)) < 1e-12
    assert abs(rx.mean()) < 1e-15 and abs(ry.mean()) < 1e-15
    # real input, real output: the Nyquist rows and columns carry nothing
    fx = np.fft.fft2(rx)
    assert np.max(np.abs(fx[:, 16])) < 1e-12 and np.max(np.abs(fx[8, :])) < 1e-12


def test_renormalise():
    rng = np.random.default_rng(4)
    vx, vy, wx, wy = rng.standard_normal((4, 8, 8))
    ox, oy = renormalise(vx, vy, wx, wy)
    assert np.sum(ox ** 2 + oy ** 2) == pytest.approx(np.sum(vx ** 2 + vy ** 2), rel=1e-14)
    assert np.allclose(ox * wy, oy * wx)  # direction kept
    z = np.zeros((8, 8))
    assert np.all(renormalise(z, z, z, z)[0] == 0.0)


def test_velocity_rms_and_vorticity():
    g = Granulation(32, 32, 1.0, 1.0, GP)
    g.update(0.0, *_draws(32, 32, 7))
    vx, vy = g.granular_field(60.0)
    ox, oy = g.velocity(60.0)
    assert np.sum(ox ** 2 + oy ** 2) == pytest.approx(np.sum(vx ** 2 + vy ** 2), rel=1e-13)
    # f_rot > 0 adds vorticity: the output's curl exceeds the granular field's
    k = 2 * np.pi * np.fft.fftfreq(32)
    curl = lambda u, v: np.abs(1j * k[None, :] * np.fft.fft2(v) - 1j * k[:, None] * np.fft.fft2(u)).sum()
    assert curl(ox, oy) > curl(vx, vy)


def test_field_at_sampled_pixels_matches_the_map():
    g = Granulation(32, 24, 1.0, 1.25, GP)
    g.update(0.0, *_draws(32, 24, 9))
    vx, vy = g.granular_field(50.0)
    pix = [(0, 0), (5, 31), (23, 7), (12, 12)]
    got = g.granular_field_at(50.0, pix)
    for n, (j, i) in enumerate(pix):
        assert got[n, 0] == pytest.approx(vx[j, i], rel=1e-12, abs=1e-15)
        assert got[n, 1] == pytest.approx(vy[j, i], rel=1e-12, abs=1e-15)


def test_population_over_updates():
    # every update leaves a full packing; a granule keeps its centre and
    # parameters from birth to death, is born at an update time and is gone
    # after t0 + 2 t_max
    nx, ny = 32, 24
    g = Granulation(nx, ny, 1.0, 1.0, GP)
    seen = {}
    deaths = 0
    for u, t in enumerate(np.arange(0.0, 600.0, 40.0)):
        before = dict(g.live)
        g.update(float(t), *_draws(nx, ny, 100 + u))
        deaths += sum(1 for c in before if c not in g.live)
        c = np.array(list(g.live.keys()))
        for j in range(ny):
            for i in range(nx):
                assert np.min(g._dist2(j, i, c[:, 0], c[:, 1])) < GP.r_inner ** 2
        for key, v in g.live.items():
            if key in seen and seen[key][0] == v[0]:
                assert seen[key] == v  # unchanged while alive
            else:
                assert v[0] == t       # a new granule is born now
            seen[key] = v
            assert t - v[0] - v[3] <= v[3]
    assert deaths > 0
