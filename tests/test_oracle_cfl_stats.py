"""Closed-form pins of the oracle's CFL time step and global diagnostics.

The CFL rule (advective limit with the fast-mode speed, diffusive limit with
the largest diffusivity of the cell, Sect. 4.3's swamp weight) and the energy,
mass and flux sums are checked on states whose answer is known on paper:
uniform fields, a uniform external field, single Fourier modes of A whose
discrete curl follows from the modified wavenumber of the sixth-order first
derivative, and swamp or conduction diffusivities made to dominate one at a
time.  Each expected value is written from the formula, not from the oracle.
"""
import math

import numpy as np
import pytest

import inputs
import oracle

NG = 3


def _ktilde(k, h):
    """Modified wavenumber of the sixth-order centred first derivative:
    D1 cos(k x) = -kt sin(k x), D1 sin(k x) = kt cos(k x), with
    kt h = [45 sin(kh) - 9 sin(2kh) + sin(3kh)] / 30."""
    return (45 * math.sin(k * h) - 9 * math.sin(2 * k * h) + math.sin(3 * k * h)) / (30 * h)


def _uniform(p, ux=0.0, uy=0.0, uz=0.0, rho=1.0, T=1.0):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    st = np.zeros((8, nz, ny, nx))
    st[3], st[4], st[5] = ux, uy, uz
    st[6] = math.log(rho)
    st[7] = math.log(T)
    return st


def _filled(p, st):
    return oracle.fill_ghosts(p, oracle.to_padded(st), np.full(p["nz"] + 2 * NG, st[6, 0, 0, 0]))


def _weight(z, zs, zt):
    s = min(max((z - zs) / (zt - zs), 0.0), 1.0)
    return 3 * s * s - 2 * s ** 3


# ---------------------------------------------------------------------------
# CFL: advective limit

def test_cfl_fast_mode_speed_of_a_uniform_field():
    """B = B_ext uniform, rho and T uniform and not 1: the advective limit is
    C_adv / (sqrt(gamma T + B^2/rho) sqrt(sum 1/dx_i^2)); the fast-mode term
    dominates (B^2/rho = 20 against gamma T = 3.3)."""
    b = (1.2, -0.9, 2.1)
    p = inputs.scheme_params(8, 8, 8, dx=1.5, dy=0.75, dz=1.0, bc_z=1,
                             bext_x=b[0], bext_y=b[1], bext_z=b[2],
                             eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0)
    rho, T = 0.3, 2.0
    u = _filled(p, _uniform(p, rho=rho, T=T))
    b2 = sum(c * c for c in b)
    inv2 = 1 / 1.5 ** 2 + 1 / 0.75 ** 2 + 1.0
    adv = math.sqrt(p["gamma"] * T + b2 / rho) * math.sqrt(inv2)
    dmax = max(p["nu"], p["eta"], p["diff_rho"], (p["gamma"] - 1) * p["kappa0"] * T ** 2.5 / rho)
    assert p["c_adv"] / adv < p["c_diff"] / (dmax * inv2)  # the advective limit binds
    assert oracle.cfl(p, u) == pytest.approx(p["c_adv"] / adv, rel=1e-14)


def test_cfl_fast_mode_of_a_fourier_mode_of_A():
    """A_z = a cos(k x): B_y = a kt sin(k x) (kt the modified wavenumber), so
    the largest fast-mode speed is sqrt(gamma T + (a kt)^2 / rho), reached
    where sin(k x) = +-1 (x = nx/4 on the grid for one wave per box)."""
    nx = 16
    p = inputs.scheme_params(nx, 8, 8, dx=0.5, dy=1.0, dz=1.0, bc_z=1,
                             eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0)
    a, rho, T = 0.8, 0.5, 1.5
    st = _uniform(p, rho=rho, T=T)
    k = 2 * math.pi / (nx * p["dx"])
    x = np.arange(nx) * p["dx"]
    st[2] = a * np.cos(k * x)[None, None, :]
    u = _filled(p, st)
    by = a * _ktilde(k, p["dx"])
    inv2 = 1 / 0.25 + 1 + 1
    adv = math.sqrt(p["gamma"] * T + by * by / rho) * math.sqrt(inv2)
    assert oracle.cfl(p, u) == pytest.approx(p["c_adv"] / adv, rel=1e-13)


def test_cfl_advection_terms_on_anisotropic_spacing():
    """Uniform u on dx != dy != dz: the advective rate gains
    |u_x|/dx + |u_y|/dy + |u_z|/dz (absolute values: u_x < 0 here)."""
    p = inputs.scheme_params(8, 8, 8, dx=2.0, dy=0.5, dz=1.0, bc_z=1,
                             eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0)
    ux, uy, uz, T = -0.7, 0.4, 0.3, 1.0
    u = _filled(p, _uniform(p, ux=ux, uy=uy, uz=uz, T=T))
    inv2 = 1 / 4.0 + 1 / 0.25 + 1.0
    adv = abs(ux) / 2.0 + abs(uy) / 0.5 + abs(uz) / 1.0 + math.sqrt(p["gamma"] * T) * math.sqrt(inv2)
    assert oracle.cfl(p, u) == pytest.approx(p["c_adv"] / adv, rel=1e-14)
    # a signed sum (u_x in place of |u_x|) or u_x/dy would change the step
    wrong = ux / 2.0 + abs(uy) / 0.5 + abs(uz) + math.sqrt(p["gamma"] * T) * math.sqrt(inv2)
    assert abs(oracle.cfl(p, u) * wrong / p["c_adv"] - 1) > 0.1


# ---------------------------------------------------------------------------
# CFL: diffusive limit, one diffusivity dominant at a time

def _swamp_box(**over):
    # the swamp ramps over the top 6 layers of a 12-layer box and ends above
    # it (z_t = z_top + 4), so no layer reaches w = 1: w < 1 at the top layer
    # is what tells eta_s w from eta_s
    nz = 12
    ztop = (nz - 1) * 1.0
    p = inputs.scheme_params(8, 8, nz, dx=1.0, dy=1.0, dz=1.0, bc_z=1,
                             z_swamp_start=ztop - 6.0, z_swamp_end=ztop + 4.0,
                             nu=0.01, eta=0.01, diff_rho=0.01, kappa0=0.0,
                             eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0)
    p.update(over)
    wtop = _weight(ztop, p["z_swamp_start"], p["z_swamp_end"])
    assert 0.4 < wtop < 0.9
    return p, wtop


@pytest.mark.parametrize("which", ["eta_swamp", "diffrho_swamp", "chi_swamp"])
def test_cfl_swamp_diffusivity(which):
    """D_max = max(nu, eta + eta_s w, D_rho + chi_rho w, chi_s w + ...): with
    one swamp coefficient large, the top layer's w sets the diffusive limit."""
    coef = 4.0
    p, wtop = _swamp_box(**{which: coef})
    u = _filled(p, _uniform(p))
    inv2 = 3.0
    base = {"eta_swamp": p["eta"], "diffrho_swamp": p["diff_rho"], "chi_swamp": 0.0}[which]
    dmax = base + coef * wtop
    want_dif = p["c_diff"] / (dmax * inv2)
    want_adv = p["c_adv"] / (math.sqrt(p["gamma"]) * math.sqrt(inv2))
    assert want_dif < want_adv
    assert oracle.cfl(p, u) == pytest.approx(want_dif, rel=1e-14)


def test_cfl_conduction_diffusivity():
    """Spitzer conduction (gamma - 1) kappa0 T^(5/2) / rho dominates in a
    cell of low density and high temperature; inside the swamp it adds to
    chi_s w.  Two layers differ in T and rho; the larger D_max wins."""
    p, wtop = _swamp_box(kappa0=0.02, chi_swamp=10.0)
    nz = p["nz"]
    st = _uniform(p, T=1.0, rho=1.0)
    # layer 2 (below the swamp): T = 4, rho = e^-2; top layer: T = 9, rho = e^-3
    st[6, 2], st[7, 2] = -2.0, math.log(4.0)
    st[6, nz - 1], st[7, nz - 1] = -3.0, math.log(9.0)
    u = _filled(p, st)
    g1 = p["gamma"] - 1
    d2 = g1 * 0.02 * 4.0 ** 2.5 / math.exp(-2.0)
    dtop = 10.0 * wtop + g1 * 0.02 * 9.0 ** 2.5 / math.exp(-3.0)
    assert dtop > d2
    inv2 = 3.0
    want_dif = p["c_diff"] / (dtop * inv2)
    adv = math.sqrt(p["gamma"] * 9.0) * math.sqrt(inv2)
    assert want_dif < p["c_adv"] / adv
    assert oracle.cfl(p, u) == pytest.approx(want_dif, rel=1e-13)


# ---------------------------------------------------------------------------
# diagnostics

def test_stats_uniform_flow_energies_and_mass():
    """Uniform rho, T, u: E_kin = rho |u|^2 / 2 V, E_th = rho T / (gamma - 1) V,
    mass = rho V, V = nx ny nz dx dy dz; no field, no flux."""
    p = inputs.scheme_params(8, 12, 6, dx=0.5, dy=1.5, dz=0.8, bc_z=1)
    rho, T = 2.5, 3.0
    u3 = (0.3, -0.4, 1.2)
    u = _filled(p, _uniform(p, ux=u3[0], uy=u3[1], uz=u3[2], rho=rho, T=T))
    V = 8 * 12 * 6 * 0.5 * 1.5 * 0.8
    s = oracle.stats(p, u)
    assert s[0] == pytest.approx(0.5 * rho * sum(c * c for c in u3) * V, rel=1e-13)
    assert s[1] == 0.0
    assert s[2] == pytest.approx(rho * T / (p["gamma"] - 1) * V, rel=1e-13)
    assert s[3] == pytest.approx(rho * V, rel=1e-13)
    assert s[4] == 0.0 and s[5] == 0.0 and s[6] == 0.0


def test_stats_magnetic_energy_of_fourier_modes():
    """A_z = a cos(kx x), A_x = b cos(kz z), A_y = c sin(kx x) in a triply
    periodic box: B_y = a kt_x sin(kx x) - b kt_z sin(kz z), B_z = c kt_x
    cos(kx x), B_x = 0; the cross term sums to zero over whole periods, so
    E_mag = (a^2 kt_x^2 + b^2 kt_z^2 + c^2 kt_x^2) N dV / 4."""
    nx, ny, nz = 16, 8, 12
    p = inputs.scheme_params(nx, ny, nz, dx=0.5, dy=1.0, dz=0.75, bc_z=1)
    a, b, c = 0.6, 0.9, 0.4
    kx = 2 * math.pi * 2 / (nx * p["dx"])
    kz = 2 * math.pi / (nz * p["dz"])
    x = np.arange(nx) * p["dx"]
    z = np.arange(nz) * p["dz"]
    st = _uniform(p)
    st[2] = a * np.cos(kx * x)[None, None, :]
    st[0] = b * np.cos(kz * z)[:, None, None]
    st[1] = c * np.sin(kx * x)[None, None, :]
    u = _filled(p, st)
    tx, tz = _ktilde(kx, p["dx"]), _ktilde(kz, p["dz"])
    N = nx * ny * nz
    dV = p["dx"] * p["dy"] * p["dz"]
    s = oracle.stats(p, u)
    assert s[1] == pytest.approx((a * a * tx * tx + b * b * tz * tz + c * c * tx * tx) * N * dV / 4,
                                 rel=1e-13)
    assert s[6] < 1e-13


def test_stats_photospheric_flux_of_a_two_polarity_plane():
    """B_z(k = 0) = B_ext,z + c kt_x cos(kx x) (1 + h): a positive and a
    negative polarity band over a uniform background.  Net flux =
    B_ext,z nx ny dx dy; unsigned flux = sum |B_z| dx dy over the photospheric
    layer only (A_y grows with height by the factor 1 + h cos(kz z), so
    another layer's flux differs)."""
    nx, ny, nz = 16, 8, 12
    bz0 = 0.3
    p = inputs.scheme_params(nx, ny, nz, dx=0.5, dy=1.25, dz=1.0, bc_z=1, bext_z=bz0)
    c, h = 0.5, 0.6
    kx = 2 * math.pi / (nx * p["dx"])
    kz = 2 * math.pi / (nz * p["dz"])
    x = np.arange(nx) * p["dx"]
    z = np.arange(nz) * p["dz"]
    st = _uniform(p)
    st[1] = c * np.sin(kx * x)[None, None, :] * (1 + h * np.cos(kz * z))[:, None, None]
    u = _filled(p, st)
    # the photospheric layer z = 0: cos(kz z) = 1
    bz = bz0 + c * _ktilde(kx, p["dx"]) * (1 + h) * np.cos(kx * x)
    assert bz.min() < 0 < bz.max()
    dA = p["dx"] * p["dy"]
    s = oracle.stats(p, u)
    assert s[4] == pytest.approx(bz0 * nx * ny * dA, rel=1e-12)
    assert s[5] == pytest.approx(ny * np.abs(bz).sum() * dA, rel=1e-13)


def _two_harmonics(n, h, amp):
    """f(s) = a1 sin(k s) + a2 sin(2 k s) on n points of spacing h (one
    period per box) and its sixth-order derivative a1 kt(k) cos(k s) +
    2-harmonic term; cos s + cos 2s has max 2 and min -9/8, so the sign of
    the derivative shows in max |B_ext + D1 f|."""
    k = 2 * math.pi / (n * h)
    s = np.arange(n) * h
    f = amp[0] * np.sin(k * s) + amp[1] * np.sin(2 * k * s)
    df = amp[0] * _ktilde(k, h) * np.cos(k * s) + amp[1] * _ktilde(2 * k, h) * np.cos(2 * k * s)
    return f, df


def test_cfl_and_flux_see_the_sign_of_each_curl_term():
    """A_x = P(y) + Q(z), A_y = R(x) + S(z), A_z = U(x) + V(y) with two
    harmonics each, over a uniform B_ext: B = (B_ext,x + V' - S',
    B_ext,y + Q' - U', B_ext,z + R' - P') with ' the sixth-order D1.  The
    largest fast-mode speed (CFL) and the unsigned photospheric flux are
    evaluated from this closed form on the grid; both depend on the sign of
    every curl term relative to B_ext, since no derivative here has a
    symmetric distribution."""
    nx, ny, nz = 16, 12, 8
    p = inputs.scheme_params(nx, ny, nz, dx=0.5, dy=0.75, dz=1.0, bc_z=1,
                             bext_x=0.4, bext_y=-0.3, bext_z=0.25,
                             eta_swamp=0.0, chi_swamp=0.0, diffrho_swamp=0.0)
    P, dP = _two_harmonics(ny, p["dy"], (0.10, 0.05))
    Q, dQ = _two_harmonics(nz, p["dz"], (0.20, 0.12))
    R, dR = _two_harmonics(nx, p["dx"], (0.07, 0.04))
    S, dS = _two_harmonics(nz, p["dz"], (0.15, -0.10))
    U, dU = _two_harmonics(nx, p["dx"], (-0.06, 0.05))
    V, dV = _two_harmonics(ny, p["dy"], (0.09, 0.06))
    rho, T = 0.4, 1.2
    st = _uniform(p, rho=rho, T=T)
    st[0] = P[None, :, None] + Q[:, None, None]
    st[1] = R[None, None, :] + S[:, None, None]
    st[2] = U[None, None, :] + V[None, :, None]
    u = _filled(p, st)
    bx = p["bext_x"] + dV[None, :, None] - dS[:, None, None]
    by = p["bext_y"] + dQ[:, None, None] - dU[None, None, :]
    bz = p["bext_z"] + dR[None, None, :] - dP[None, :, None]
    b2full = bx ** 2 + by ** 2 + bz ** 2  # broadcasts to (nz, ny, nx)
    b2 = b2full.max()
    inv2 = 1 / 0.25 + 1 / 0.5625 + 1.0
    adv = math.sqrt(p["gamma"] * T + b2 / rho) * math.sqrt(inv2)
    assert oracle.cfl(p, u) == pytest.approx(p["c_adv"] / adv, rel=1e-13)
    s = oracle.stats(p, u)
    dA = p["dx"] * p["dy"]
    assert s[4] == pytest.approx(p["bext_z"] * nx * ny * dA, rel=1e-12)
    assert s[5] == pytest.approx(np.abs(bz[0]).sum() * dA, rel=1e-13)
    # E_mag of the same field: the cross terms of the harmonics vanish
    dVol = dA * p["dz"]
    assert s[1] == pytest.approx(0.5 * b2full.sum() * dVol, rel=1e-13)
