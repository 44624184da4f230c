"""Pins of the oracle's ghost-zone rules, potential-field extrapolation,
magnetogram inversion, swamp weight and geometry, against closed forms and
invariants fixed by the paper and by the mathematics."""
import os

import numpy as np
import pytest

import inputs
import oracle

NG = oracle.NG
HERE = os.path.dirname(os.path.abspath(__file__))


def _params(nx, ny, nz, **over):
    p = inputs.scheme_params(nx, ny, nz)
    p.update(over)
    return p


def test_isothermal_hydrostatic_is_fixed_point_of_ghost_rules():
    """Sect. 2.5 Eq. 8 (bottom T) and Sect. 4.1 Eqs. 11, 13 (top T, rho): an
    exactly isothermal hydrostatic column, rho ~ exp(g_z z / T), must be
    reproduced in the ghost layers (catches a sign of g, a spurious 1/gamma
    or a wrong distance)."""
    nx, ny, nz = 8, 8, 12
    T0, gz = 2.0, -0.2
    p = _params(nx, ny, nz, gz=gz)
    k = np.arange(-NG, nz + NG)
    lnrho_exact = 0.3 + gz * k * p["dz"] / T0
    st = np.zeros((8, nz, ny, nx))
    st[6] = lnrho_exact[NG:NG + nz, None, None]
    st[7] = np.log(T0)
    u = oracle.to_padded(st)
    oracle.fill_ghosts(p, u, lnrho_exact)
    lnT = u[7, :, NG:-NG, NG:-NG]
    lnr = u[6, :, NG:-NG, NG:-NG]
    assert np.allclose(lnT, np.log(T0), rtol=0, atol=1e-14)
    assert np.allclose(lnr, lnrho_exact[:, None, None], rtol=0, atol=1e-13)


def test_bottom_temperature_is_hydrostatic_for_any_profile():
    """Eq. 8: with rho fixed below the photosphere, T in the ghost layers
    makes p = rho T hydrostatic between consecutive layers:
    p_j / p_{j+1} = exp(|g_z| dz / T_{j+1}); the pressure grows downward."""
    nx, ny, nz = 8, 8, 10
    p = _params(nx, ny, nz)
    case = inputs.make_box(nx, ny, nz, seed=3)
    rng = np.random.default_rng(1)
    st = case.state.copy()
    st[7] += 0.1 * rng.standard_normal(st[7].shape)
    u = oracle.to_padded(st)
    oracle.fill_ghosts(p, u, case.lnrho0)
    lnp = u[6] + u[7]
    for m in range(1, NG + 1):
        kj, kj1 = NG - m, NG - m + 1
        ratio = lnp[kj] - lnp[kj1]
        assert np.all(ratio > 0)
        assert np.allclose(ratio, -p["gz"] * p["dz"] / np.exp(u[7, kj1]), rtol=1e-12, atol=0)
    # density below and at the photosphere: the initial profile ('fg')
    for m in range(1, NG + 1):
        assert np.all(u[6, NG - m] == case.lnrho0[NG - m])


def test_velocity_ghost_symmetries():
    """Closed bottom and top (Sect. 2.5, 4): u_z antisymmetric about the
    boundary layers; u_hor symmetric at the top; the stateful u_hor ghosts
    below the photosphere (Eq. 5) are not overwritten by the ghost fill."""
    nx, ny, nz = 8, 8, 10
    p = _params(nx, ny, nz)
    case = inputs.make_box(nx, ny, nz, seed=2)
    rng = np.random.default_rng(5)
    st = case.state.copy()
    st[3:6] = rng.standard_normal(st[3:6].shape)
    u = oracle.to_padded(st)
    u[3:5, :NG] = rng.standard_normal(u[3:5, :NG].shape)
    keep = u[3:5, :NG, NG:-NG, NG:-NG].copy()
    oracle.fill_ghosts(p, u, case.lnrho0)
    kb, kt = NG, NG + nz - 1
    for m in range(1, NG + 1):
        assert np.array_equal(u[5, kb - m], -u[5, kb + m])
        assert np.array_equal(u[5, kt + m], -u[5, kt - m])
        assert np.array_equal(u[3:5, kt + m], u[3:5, kt - m])
        assert np.array_equal(u[7, kt + m], u[7, kt - m])
    assert np.array_equal(u[3:5, :NG, NG:-NG, NG:-NG], keep)


def test_periodic_rims():
    nx, ny, nz = 8, 16, 9
    p = _params(nx, ny, nz)
    case = inputs.make_box(nx, ny, nz, seed=4)
    u = oracle.to_padded(case.state)
    oracle.fill_ghosts(p, u, case.lnrho0)
    core = u[:, :, NG:NG + ny, NG:NG + nx]
    wrapped = np.pad(core, ((0, 0), (0, 0), (NG, NG), (NG, NG)), mode="wrap")
    assert np.array_equal(u, wrapped)


@pytest.mark.parametrize("mx,my", [(3, 0), (0, 2), (2, 5), (16, 0), (4, 8)])
def test_pfe_single_mode(mx, my):
    """Eq. 17: a single Fourier mode of A decays as exp(-|k| Delta''z) into
    the top ghosts, Delta''z = j dz; below the photosphere the inverted
    extrapolation grows it as exp(+f_b |k| j dz) with f_b = 0.2 (Sect. 2.4)."""
    nx, ny, nz = 32, 16, 8
    dx, dy, dz = 1.0, 2.0, 0.7
    p = _params(nx, ny, nz, dx=dx, dy=dy, dz=dz)
    x = np.arange(nx)[None, :] * dx
    y = np.arange(ny)[:, None] * dy
    kx, ky = 2 * np.pi * mx / (nx * dx), 2 * np.pi * my / (ny * dy)
    mode = np.cos(kx * x + ky * y + 0.4)
    kk = np.hypot(kx, ky)
    st = np.zeros((8, nz, ny, nx))
    st[6] = 0.0
    st[7] = 0.0
    for c in range(3):
        st[c, nz - 1] = (c + 1) * mode
        st[c, 0] = (2 - c) * mode
    u = oracle.to_padded(st)
    oracle.fill_ghosts(p, u, np.zeros(nz + 2 * NG))
    for c in range(3):
        for m in range(1, NG + 1):
            top = u[c, NG + nz - 1 + m, NG:-NG, NG:-NG]
            bot = u[c, NG - m, NG:-NG, NG:-NG]
            assert np.allclose(top, (c + 1) * mode * np.exp(-kk * m * dz), rtol=0, atol=1e-12)
            assert np.allclose(bot, (2 - c) * mode * np.exp(0.2 * kk * m * dz), rtol=0, atol=1e-12)


def test_ghost_fill_fft_variant_matches_plain_dft():
    """The numpy-FFT ghost fill used for large planes equals the plain-DFT
    one (every ghost cell, all fields)."""
    case = inputs.make_box(16, 32, 10, seed=12, dx=2.0, dy=0.5)
    a = oracle.to_padded(case.state)
    b = a.copy()
    oracle.fill_ghosts(case.params, a, case.lnrho0, pfe="dft")
    oracle.fill_ghosts(case.params, b, case.lnrho0, pfe="fft")
    assert np.allclose(a, b, rtol=0, atol=1e-12)


def test_pfe_plain_dft_matches_numpy_fft():
    rng = np.random.default_rng(0)
    nx, ny = 16, 32
    plane = rng.standard_normal((ny, nx))
    zf = [-0.5, -1.0, 0.2]
    a = oracle.pfe_plane(nx, ny, 16.0, 64.0, plane, zf)
    b = oracle.pfe_plane_fft(16.0, 64.0, plane, zf)
    assert np.allclose(a, b, rtol=0, atol=1e-12)
    # zero distance is the identity; the mean (k = 0) passes unchanged
    c = oracle.pfe_plane(nx, ny, 16.0, 64.0, plane, [0.0])
    assert np.allclose(c[0], plane, rtol=0, atol=1e-13)
    assert np.isclose(a[0].mean(), plane.mean(), rtol=0, atol=1e-14)


def _d1_periodic(p, plane2d, axis):
    ny, nx = plane2d.shape
    q = dict(p, nz=1, bc_z=1)
    u = np.zeros((8, 1 + 2 * NG, ny + 2 * NG, nx + 2 * NG))
    u[0] = np.pad(plane2d[None], ((NG, NG), (NG, NG), (NG, NG)), mode="wrap")
    return oracle.deriv(q, u, 0, 0, axis)[0]


def test_a_target_reproduces_band_limited_bz():
    """Eq. 7: B_z = d_x A_y - d_y A_x.  With the discrete first derivative the
    inversion reproduces B_z exactly up to the four modes whose modified
    wavenumber vanishes (mean and Nyquist)."""
    nx, ny = 32, 16
    p = _params(nx, ny, 4, dx=1.0, dy=1.5)
    rng = np.random.default_rng(7)
    bz = rng.standard_normal((ny, nx))
    ax, ay = oracle.a_target(p, bz)
    curl = _d1_periodic(p, ay, 0) - _d1_periodic(p, ax, 1)
    h = np.fft.fft2(bz)
    for (b, a) in [(0, 0), (0, nx // 2), (ny // 2, 0), (ny // 2, nx // 2)]:
        h[b, a] = 0.0
    band = np.real(np.fft.ifft2(h))
    assert np.allclose(curl, band, rtol=0, atol=1e-12)


def test_a_target_fft_variant_matches_plain_dft():
    nx, ny = 32, 16
    p = _params(nx, ny, 4, dx=1.0, dy=1.5)
    bz = np.random.default_rng(8).standard_normal((ny, nx))
    a = oracle.a_target(p, bz)
    b = oracle.a_target_fft(p, bz)
    assert np.allclose(a[0], b[0], rtol=0, atol=1e-13) and np.allclose(a[1], b[1], rtol=0, atol=1e-13)


def test_swamp_weight():
    """Sect. 4.3: w = 0 below z_s, 1 above z_t, cubic step with zero slope at
    both ends, monotone in between."""
    p = _params(8, 8, 40)
    zs, zt = p["z_swamp_start"], p["z_swamp_end"]
    assert oracle.swamp_weight(p, zs - 1.0) == (0.0, 0.0)
    assert oracle.swamp_weight(p, zs) == (0.0, 0.0)
    assert oracle.swamp_weight(p, zt) == (1.0, 0.0)
    assert oracle.swamp_weight(p, zt + 2.0) == (1.0, 0.0)
    w, wp = oracle.swamp_weight(p, 0.5 * (zs + zt))
    assert abs(w - 0.5) < 1e-15 and abs(wp - 1.5 / (zt - zs)) < 1e-15
    zz = np.linspace(zs, zt, 101)
    ws = np.array([oracle.swamp_weight(p, z)[0] for z in zz])
    assert np.all(np.diff(ws) >= 0)
    # slope vanishes at both ends and matches a centred difference inside
    for z in (zs + 1e-6, zt - 1e-6):
        assert abs(oracle.swamp_weight(p, z)[1]) < 1e-5
    z = zs + 0.3 * (zt - zs)
    fd = (oracle.swamp_weight(p, z + 1e-6)[0] - oracle.swamp_weight(p, z - 1e-6)[0]) / 2e-6
    assert abs(fd - oracle.swamp_weight(p, z)[1]) < 1e-8


def test_div_b_vanishes_to_roundoff():
    """Eq. 6: B = curl A is divergence free; the discrete D1 operators commute,
    so max |div B| stays at roundoff for an arbitrary A."""
    nx, ny, nz = 16, 8, 12
    p = _params(nx, ny, nz, bc_z=1)
    rng = np.random.default_rng(11)
    st = np.zeros((8, nz, ny, nx))
    st[0:3] = rng.standard_normal((3, nz, ny, nx))
    u = oracle.to_padded(st)
    oracle.fill_ghosts(p, u, np.zeros(nz + 2 * NG))
    s = oracle.stats(p, u)
    assert s[6] < 1e-13


def test_table1_storage_geometry():
    """Sect. 5.3, Table 1: the 17 GB snapshot and the +31 % / +16 % storage
    overheads follow from 8 double-precision fields with three ghost layers
    on every side (pins the ghost width and field count used here)."""
    g = {}
    for line in open(os.path.join(HERE, "golden", "table1_storage.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, val = line.split()
        g[key] = float(val)
    nx, ny, nz = int(g["nx"]), int(g["ny"]), int(g["nz"])
    px, py, pz = int(g["nprocx"]), int(g["nprocy"]), int(g["nprocz"])
    nf, ng = inputs.NFIELD, oracle.NG
    assert ng == inputs.NGHOST
    mono = nf * (nx + 2 * ng) * (ny + 2 * ng) * (nz + 2 * ng) * g["bytes_per_value"]
    assert round(mono / 1e9) in (g["snapshot_gb"], g["snapshot_gb"] + 1)
    assert abs(mono / 1e9 - g["snapshot_gb"]) < 1.0
    dist = px * py * pz * (nx // px + 2 * ng) * (ny // py + 2 * ng) * (nz // pz + 2 * ng)
    over_dist = dist / ((nx + 2 * ng) * (ny + 2 * ng) * (nz + 2 * ng)) - 1.0
    assert round(100 * over_dist) == g["io_dist_overhead_percent"]
    cxy = pz * (nx + 2 * ng) * (ny + 2 * ng) * (nz // pz + 2 * ng)
    over_cxy = cxy / ((nx + 2 * ng) * (ny + 2 * ng) * (nz + 2 * ng)) - 1.0
    assert round(100 * over_cxy) == g["io_collect_xy_overhead_percent"]


def test_generated_magnetograms_are_flux_balanced():
    """Sect. 2.1: the driving magnetograms are flux balanced."""
    for name in ("spots4_32x32x32", "bipoles8_64x64x64"):
        c = inputs.make_case(name)
        assert abs(c.bz.sum()) < 1e-12 * np.abs(c.bz).sum()
        assert np.abs(c.bz).max() > 0.1
        # photospheric plasma beta 2 p / B^2 (p = 1) near or above unity
        assert 2.0 / np.abs(c.bz).max() ** 2 > 0.8
