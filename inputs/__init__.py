"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

This module holds no step of the method: no stencil, boundary rule, Fourier
multiplier of the potential-field boundary, CFL rule or time integrator.  It
builds the things a run *starts from*: scheme constants, photospheric
magnetograms, driver velocity snapshots, and an initial hydrostatic,
potential-field state.  Both sides read these arrays; neither side's output
ever feeds back into them.

Workloads (synthetic stand-ins for the paper's Hinode-driven active-region run,
Sect. 2.1 and 5.3: 1024 x 1024 horizontal points, three ghost layers):

* ``spots4_32x32x32``       4 Gaussian spots (sigma 3 cells, +-1), 50 RK3 steps
* ``bipoles40_256x256x256``  40 bipoles, log-normal fluxes, k^-5/3 solenoidal driver
* ``ar_1024x1024x256``       400 bipoles plus a +-5 active-region pair (sigma 40
                            cells), horizontal spacing 4x vertical
* ``bipoles8_64x64x64``      8 bipoles, 100 steps (gradient workload)
* ``bipoles100_512x512x256`` 100 bipoles (checkpointed gradient workload)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Tuple

import numpy as np

NGHOST = 3
FIELDS = ("ax", "ay", "az", "ux", "uy", "uz", "lnrho", "lnTT")
NFIELD = len(FIELDS)

# Scheme constants in code units (mu0 = 1, R/mu = 1).  The paper gives the
# physical values tau_u = 0.5 s^-1 (Sect. 2.3), D_rho = 8e6 m^2/s (Sect. 2.5)
# and fbcz_bot = 0.2 (Sect. 2.4); it gives no code-unit values, so these are
# the frozen proposal of the scheme.
PARAM_DEFAULTS = dict(
    gamma=5.0 / 3.0,
    gz=-0.2,
    nu=0.05,
    eta=0.05,
    kappa0=2e-8,
    diff_rho=0.05,
    eta_swamp=0.5,
    chi_swamp=0.5,
    diffrho_swamp=0.5,
    tau_u=0.5,
    tau_A=0.5,
    t_ramp=0.5,
    f_pfe_bottom=0.2,
    c_adv=0.4,
    c_diff=0.25,
    dt_fixed=0.0,
    bext_x=0.0,
    bext_y=0.0,
    bext_z=0.0,
    bc_z=0,
    # Newtonian cooling (Sect. 3.1): off in every named workload
    nc_tau=0.0,
    nc_lnrho_magn=8.0,
    nc_lnrho_width=2.0,
)


def scheme_params(nx: int, ny: int, nz: int, dx: float = 1.0, dy: float = 1.0,
                  dz: float = 1.0, swamp_cells: int = 4, **over) -> Dict:
    """Parameter dict of one box; the swamp spans the top `swamp_cells` cells."""
    p = dict(PARAM_DEFAULTS)
    ztop = (nz - 1) * dz
    p.update(nx=int(nx), ny=int(ny), nz=int(nz), dx=float(dx), dy=float(dy),
             dz=float(dz), z_swamp_start=ztop - swamp_cells * dz,
             z_swamp_end=ztop, nc_z_max=10.0 * dz, nc_z_width=1.0 * dz)
    p.update(over)
    return p


# --------------------------------------------------------------------------
# magnetograms

def _periodic_gauss(nx, ny, x0, y0, sigma):
    """Gaussian of width sigma (cells) summed over the nearest periodic images
    (evaluated within 8 sigma of the centre; beyond that it is below 1e-13)."""
    g = np.zeros((ny, nx))
    w = int(np.ceil(8.0 * sigma))
    if 2 * w + 1 >= min(nx, ny):
        x = np.arange(nx)[None, :]
        y = np.arange(ny)[:, None]
        for sx in (-1, 0, 1):
            for sy in (-1, 0, 1):
                r2 = (x - x0 - sx * nx) ** 2 + (y - y0 - sy * ny) ** 2
                g += np.exp(-r2 / (2.0 * sigma * sigma))
        return g
    ic, jc = int(np.floor(x0)), int(np.floor(y0))
    xi = np.arange(ic - w, ic + w + 1)
    yj = np.arange(jc - w, jc + w + 1)
    vals = np.exp(-((yj[:, None] - y0) ** 2 + (xi[None, :] - x0) ** 2) / (2.0 * sigma * sigma))
    np.add.at(g, (yj[:, None] % ny, xi[None, :] % nx), vals)
    return g


def flux_balance(bz: np.ndarray) -> np.ndarray:
    """Rescale each polarity by a constant so that the net flux vanishes.

    Sect. 2.1: both polarities are rescaled separately by a constant factor to
    obtain a flux-balanced magnetogram (the box is periodic horizontally).
    """
    pos = bz[bz > 0].sum()
    neg = -bz[bz < 0].sum()
    if pos == 0.0 or neg == 0.0:
        return bz.copy()
    mean = 0.5 * (pos + neg)
    out = bz.copy()
    out[bz > 0] *= mean / pos
    out[bz < 0] *= mean / neg
    return out


def magnetogram_spots(nx, ny, n_spots, sigma, seed):
    """n_spots Gaussian spots of alternating sign +-1 at seeded positions."""
    rng = np.random.default_rng(seed)
    bz = np.zeros((ny, nx))
    for s in range(n_spots):
        x0, y0 = rng.uniform(0, nx), rng.uniform(0, ny)
        bz += (1.0 if s % 2 == 0 else -1.0) * _periodic_gauss(nx, ny, x0, y0, sigma)
    return flux_balance(bz)


BIPOLE_PEAK = 0.3


def magnetogram_bipoles(nx, ny, n_bipoles, seed, sigma=3.0, sep=(4.0, 16.0),
                        ar_pair: Optional[Tuple[float, float, float]] = None):
    """Bipoles with log-normal fluxes (mu 0, sigma 1; the flux unit is that of
    a pole with peak |B_z| = BIPOLE_PEAK), separations uniform in
    `sep` cells, uniform orientation and centre; optional active-region pair
    (amplitude, sigma, separation in cells) at the centre of the box."""
    rng = np.random.default_rng(seed)
    bz = np.zeros((ny, nx))
    for _ in range(n_bipoles):
        flux = rng.lognormal(0.0, 1.0)
        d = rng.uniform(*sep)
        th = rng.uniform(0.0, 2.0 * math.pi)
        xc, yc = rng.uniform(0, nx), rng.uniform(0, ny)
        # the median pole peaks at |B_z| = 0.3: with p = 1 at the photosphere
        # even the strongest of 40 log-normal poles keeps plasma beta >~ 1
        # (Sect. 2.1: beta is near or above unity in the photosphere); a
        # 4x stronger unit drove grid-scale growth at the strongest pole
        amp = BIPOLE_PEAK * flux
        dx, dy = 0.5 * d * math.cos(th), 0.5 * d * math.sin(th)
        bz += amp * _periodic_gauss(nx, ny, (xc + dx) % nx, (yc + dy) % ny, sigma)
        bz -= amp * _periodic_gauss(nx, ny, (xc - dx) % nx, (yc - dy) % ny, sigma)
    if ar_pair is not None:
        a, s, d = ar_pair
        bz += a * _periodic_gauss(nx, ny, nx / 2 - d / 2, ny / 2, s)
        bz -= a * _periodic_gauss(nx, ny, nx / 2 + d / 2, ny / 2, s)
    return flux_balance(bz)


# --------------------------------------------------------------------------
# driver velocity snapshots

def _int_wavenumbers(nx, ny):
    kx = np.fft.fftfreq(nx, d=1.0 / nx)[None, :]
    ky = np.fft.fftfreq(ny, d=1.0 / ny)[:, None]
    return kx, ky


def driver_smoothed_noise(nx, ny, sigma, rms, seed):
    """Per-cell N(0,1) horizontal velocity, periodic Gaussian smoothing of width
    sigma cells, scaled to the given rms of |v_hor|.  Returns (2, ny, nx)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((2, ny, nx))
    kx, ky = _int_wavenumbers(nx, ny)
    k2 = (2 * np.pi * kx / nx) ** 2 + (2 * np.pi * ky / ny) ** 2
    filt = np.exp(-0.5 * k2 * sigma * sigma)
    v = np.real(np.fft.ifft2(np.fft.fft2(v) * filt))
    v *= rms / math.sqrt(np.mean(v[0] ** 2 + v[1] ** 2))
    return v


def driver_solenoidal(nx, ny, kmax, rms, seed, slope=-5.0 / 3.0):
    """Random solenoidal v = (d_y psi, -d_x psi) with shell spectrum E(k) ~
    k^slope for 1 <= |k| <= kmax (integer wavenumbers), random phases, scaled
    to the given rms.  Returns (2, ny, nx)."""
    rng = np.random.default_rng(seed)
    kx, ky = _int_wavenumbers(nx, ny)
    kk = np.sqrt(kx ** 2 + ky ** 2)
    amp = np.zeros_like(kk)
    sel = (kk >= 1.0) & (kk <= kmax)
    # |v^|^2 ~ E(k)/k in 2D, and |psi^| = |v^|/k
    amp[sel] = kk[sel] ** ((slope - 1.0) / 2.0) / kk[sel]
    phase = rng.uniform(0.0, 2.0 * np.pi, size=kk.shape)
    psi_h = amp * np.exp(1j * phase)
    vx = np.real(np.fft.ifft2(1j * (2 * np.pi * ky / ny) * psi_h))
    vy = np.real(np.fft.ifft2(-1j * (2 * np.pi * kx / nx) * psi_h))
    v = np.stack([vx, vy])
    v *= rms / math.sqrt(np.mean(v[0] ** 2 + v[1] ** 2))
    return v


# --------------------------------------------------------------------------
# initial state

def initial_atmosphere(nz, dz, gz, t_bottom=1.0, t_top=100.0, zc_cells=12.0,
                       width_cells=2.0, z=None):
    """ln T0 and ln rho0 on k = -3 .. nz+2.

    T0(z) = T_b + (T_t - T_b)/2 (1 + tanh((z - z_c)/w)), z_c = zc_cells dz,
    w = width_cells dz; ln p from trapezoid hydrostatics, ln p_{k+1} = ln p_k
    + (z_{k+1} - z_k) g_z (1/T_k + 1/T_{k+1})/2 with p = 1 at z = 0; ln rho0 =
    ln p - ln T0 (p = rho T).  z: the layer positions (nz + 6, a
    non-uniform grid); default z_k = k dz."""
    k = np.arange(-NGHOST, nz + NGHOST)
    z = k * dz if z is None else np.asarray(z, dtype=np.float64)
    T = t_bottom + (t_top - t_bottom) * 0.5 * (1.0 + np.tanh((z - zc_cells * dz) / (width_cells * dz)))
    lnp = np.zeros_like(z)
    k0 = NGHOST
    for q in range(k0 + 1, len(z)):
        lnp[q] = lnp[q - 1] + (z[q] - z[q - 1]) * gz * 0.5 * (1.0 / T[q - 1] + 1.0 / T[q])
    for q in range(k0 - 1, -1, -1):
        lnp[q] = lnp[q + 1] - (z[q + 1] - z[q]) * gz * 0.5 * (1.0 / T[q + 1] + 1.0 / T[q])
    return np.log(T), lnp - np.log(T)


def stretched_z(nz, dz_bottom, dz_top, k_c, width):
    """Positions of the layers k = -3 .. nz+2 of a vertical grid whose
    spacing rises smoothly from dz_bottom to dz_top around layer k_c (the
    production grid goes from about 100 km to about 800 km, Sect. 1):
    z'(k) = dz_b + (dz_t - dz_b) (1 + tanh((k - k_c)/width)) / 2, integrated
    in closed form, z(0) = 0.  Returns (z, z'(k), z''(k))."""
    k = np.arange(-NGHOST, nz + NGHOST, dtype=np.float64)
    d = dz_top - dz_bottom
    lc = lambda x: np.log(np.cosh(x))
    z = dz_bottom * k + 0.5 * d * (k + width * (lc((k - k_c) / width) - lc(-k_c / width)))
    zp = dz_bottom + 0.5 * d * (1.0 + np.tanh((k - k_c) / width))
    zpp = 0.5 * d / width / np.cosh((k - k_c) / width) ** 2
    return z, zp, zpp


def initial_potential_field(bz, nz, dx, dy, dz, dtype=np.float64, z=None):
    """Potential field whose vertical component at z = 0 is bz, as a vector
    potential in the Weyl gauge with A_z = 0, using exact spectral wavenumbers:
    A^(k, z) = (i k_y, -i k_x, 0) B^_z(k) / |k|^2 exp(-|k| z) for k = 0..nz-1,
    at z = k dz or, with z (the nz + 6 layer positions of a non-uniform grid),
    at the positions of the interior layers.
    (Initial-condition preparation; not the library's own inversion.)"""
    ny, nx = bz.shape
    kx = 2 * np.pi * np.fft.rfftfreq(nx, d=dx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=dy)[:, None]
    kk = np.sqrt(kx ** 2 + ky ** 2)
    bh = np.fft.rfft2(bz)
    bh[0, 0] = 0.0
    if nx % 2 == 0:
        bh[:, nx // 2] = 0.0
    if ny % 2 == 0:
        bh[ny // 2, :] = 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        axh = np.where(kk > 0, 1j * ky * bh / kk ** 2, 0.0)
        ayh = np.where(kk > 0, -1j * kx * bh / kk ** 2, 0.0)
    ax = np.empty((nz, ny, nx), dtype=dtype)
    ay = np.empty((nz, ny, nx), dtype=dtype)
    zi = np.arange(nz) * dz if z is None else np.asarray(z, dtype=np.float64)[NGHOST:NGHOST + nz]
    for k in range(nz):
        dec = np.exp(-kk * zi[k])
        ax[k] = np.fft.irfft2(axh * dec, s=(ny, nx))
        ay[k] = np.fft.irfft2(ayh * dec, s=(ny, nx))
    return ax, ay, np.zeros((nz, ny, nx), dtype=dtype)


@dataclasses.dataclass
class Case:
    name: str
    params: Dict
    state: np.ndarray          # (8, nz, ny, nx) interior, float64
    lnrho0: np.ndarray         # (nz + 6,) k = -3 .. nz+2
    lnT0: np.ndarray           # (nz + 6,) initial ln T stratification
    bz: np.ndarray             # (ny, nx) photospheric target
    v0: np.ndarray             # (2, ny, nx) driver snapshot at t0
    v1: np.ndarray             # (2, ny, nx) driver snapshot at t1
    t0: float
    t1: float
    nsteps: int


def make_box(nx, ny, nz, seed=0, magnetogram="spots", n_mag=4, sigma=3.0,
             driver="noise", driver_rms=0.01, dx=1.0, dy=1.0, dz=1.0,
             nsteps=50, name=None, ar_pair=None, t1=1.0, dtype=np.float64, bz_scale=1.0, z=None,
             **over) -> Case:
    """z: the nz + 6 layer positions of a non-uniform vertical grid (p["z"]);
    the swamp then spans the top four local spacings and the atmosphere and
    the potential field are evaluated at the positions (dz stays the scale
    of the temperature transition)."""
    p = scheme_params(nx, ny, nz, dx, dy, dz, **over)
    if z is not None:
        z = np.asarray(z, dtype=np.float64)
        ztop = z[NGHOST + nz - 1]
        p.update(z=z, z_swamp_start=ztop - 4.0 * (ztop - z[NGHOST + nz - 2]), z_swamp_end=ztop)
        p.update(over)
    if magnetogram == "spots":
        bz = magnetogram_spots(nx, ny, n_mag, sigma, seed)
    else:
        bz = magnetogram_bipoles(nx, ny, n_mag, seed, sigma=sigma, ar_pair=ar_pair)
    bz = bz * bz_scale
    if driver == "noise":
        v0 = driver_smoothed_noise(nx, ny, 2.0, driver_rms, seed)
        v1 = driver_smoothed_noise(nx, ny, 2.0, driver_rms, seed + 1)
    else:
        km = min(32, nx // 2, ny // 2)
        v0 = driver_solenoidal(nx, ny, km, driver_rms, seed)
        v1 = driver_solenoidal(nx, ny, km, driver_rms, seed + 1)
    lnT0, lnrho0 = initial_atmosphere(nz, dz, p["gz"], z=z)
    ax, ay, az = initial_potential_field(bz, nz, dx, dy, dz, dtype, z=z)
    st = np.zeros((NFIELD, nz, ny, nx), dtype=dtype)
    st[0], st[1], st[2] = ax, ay, az
    st[6] = lnrho0[NGHOST:NGHOST + nz, None, None]
    st[7] = lnT0[NGHOST:NGHOST + nz, None, None]
    return Case(name or f"box_{nx}x{ny}x{nz}", p, st, lnrho0, lnT0, bz, v0, v1, 0.0,
                float(t1), nsteps)


WORKLOADS = {
    "spots4_32x32x32": dict(nx=32, ny=32, nz=32, magnetogram="spots", n_mag=4,
                            driver="noise", nsteps=50),
    "bipoles40_256x256x256": dict(nx=256, ny=256, nz=256, magnetogram="bipoles",
                                  n_mag=40, driver="solenoidal", nsteps=200),
    "ar_1024x1024x256": dict(nx=1024, ny=1024, nz=256, dx=4.0, dy=4.0,
                             magnetogram="bipoles", n_mag=400,
                             ar_pair=(5.0, 40.0, 200.0), driver="solenoidal",
                             nsteps=1000),
    "bipoles8_64x64x64": dict(nx=64, ny=64, nz=64, magnetogram="bipoles",
                              n_mag=8, driver="noise", nsteps=100),
    # a third of the flux unit: with the full unit the strongest of the 100
    # log-normal poles (|B_z| = 4.7, photospheric beta 0.09) drives grid-scale
    # growth within 200 steps; at a third the box stays finite for ~800 steps
    # (then the same growth sets in), so gradients use 600 steps
    "bipoles100_512x512x256": dict(nx=512, ny=512, nz=256, magnetogram="bipoles",
                                   n_mag=100, driver="solenoidal", nsteps=600, bz_scale=1.0 / 3.0),
    # the production recipe's 1024^2 planes on 16 layers: profiler captures of
    # the potential-field FFT at full plane size with a few GB on the device
    "ar_1024x1024x16": dict(nx=1024, ny=1024, nz=16, dx=4.0, dy=4.0,
                            magnetogram="bipoles", n_mag=400,
                            ar_pair=(5.0, 40.0, 200.0), driver="solenoidal",
                            nsteps=1000),
    # the 256^3 recipe at an eighth of the volume: profiler captures of the
    # adjoint kernels (coefficient fields 0.34 GB, above the 129 MB L2)
    "bipoles20_128x128x128": dict(nx=128, ny=128, nz=128, magnetogram="bipoles",
                                  n_mag=20, driver="solenoidal", nsteps=200),
    # the 256^3 recipe's planes on 64 layers: profiler captures of the adjoint
    # kernels with the 256^2 tiling and work-item count per chunk of the
    # 256^3 box (coefficient fields 0.67 GB; about 2.5 GB on the device)
    "bipoles40_256x256x64": dict(nx=256, ny=256, nz=64, magnetogram="bipoles",
                                 n_mag=40, driver="solenoidal", nsteps=200),
}


def make_case(name: str, seed: int = 0, dtype=np.float64) -> Case:
    """A named workload; dtype sets the precision of the initial state array
    (the profiles, magnetogram and drivers stay float64)."""
    kw = dict(WORKLOADS[name])
    return make_box(seed=seed, name=name, dtype=dtype, **kw)


def padded_shape(nx, ny, nz):
    return (NFIELD, nz + 2 * NGHOST, ny + 2 * NGHOST, nx + 2 * NGHOST)


def granulation_draws(nx: int, ny: int, seed: int, update: int = 0):
    """The random inputs of one granulation-driver update: uint32 visiting
    keys and two standard normal fields (lifetime and amplitude draws),
    [ny][nx] each, from a generator seeded by (seed, update)."""
    rng = np.random.default_rng([seed, update])
    keys = rng.integers(0, 2 ** 32, (ny, nx), dtype=np.uint64).astype(np.uint32)
    return keys, rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))
