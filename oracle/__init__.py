"""FP64 CPU oracle of the driven coronal MHD step -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this package.  The product (the CUDA library and its Python binding)
never imports, loads or calls it, and it shares no code with the product: it
wraps ``mhd_oracle.c`` (plain loops, FP64), compiled here with gcc.

Array conventions: interior state (8, nz, ny, nx) float64 in field order
Ax, Ay, Az, ux, uy, uz, ln rho, ln T; the padded state adds 3 ghost cells on
every side, (8, nz+6, ny+6, nx+6), x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

NG = 3
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

_PARAM_ORDER = ("dx", "dy", "dz", "gamma", "gz", "nu", "eta", "kappa0",
                "diff_rho", "eta_swamp", "chi_swamp", "diffrho_swamp",
                "z_swamp_start", "z_swamp_end", "tau_u", "tau_A", "t_ramp",
                "f_pfe_bottom", "c_adv", "c_diff", "dt_fixed", "bext_x",
                "bext_y", "bext_z")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no fused multiply-add,
    the same sequence of roundings on x86 and Arm)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off",
                               "-std=gnu11", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.or_fill_ghosts.argtypes = [ip, dp, dp, dp]
        _lib.or_fill_ghosts_nopfe.argtypes = [ip, dp, dp, dp]
        _lib.or_set_nc_profile.argtypes = [ctypes.c_int, dp, dp]
        _lib.or_set_zgrid.argtypes = [ctypes.c_int, dp]
        _lib.or_rhs.argtypes = [ip, dp, dp, dp, dp, dp, dp, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, dp]
        _lib.or_cfl.argtypes = [ip, dp, dp]
        _lib.or_cfl.restype = ctypes.c_double
        _lib.or_stats.argtypes = [ip, dp, dp, dp]
        _lib.or_run.argtypes = [ip, dp, dp, dp, dp, dp, dp, dp, ctypes.c_double,
                                ctypes.c_double, dp, ctypes.c_int, dp]
        _lib.or_run.restype = ctypes.c_int
        _lib.or_pfe_plane.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, dp, ctypes.c_int, dp, dp]
        _lib.or_a_target.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, dp, dp, dp]
        _lib.or_deriv.argtypes = [ip, dp, dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, dp]
        _lib.or_swamp_weight.argtypes = [dp, ctypes.c_double, dp, dp]
        _lib.or_rhs_cells.argtypes = [ip, dp, dp, dp, dp, dp, dp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, ip, dp]
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(p: Dict) -> np.ndarray:
    return np.array([p["nx"], p["ny"], p["nz"], int(p.get("bc_z", 0))], dtype=np.int32)


_NC_ORDER = ("nc_tau", "nc_lnrho_magn", "nc_lnrho_width", "nc_z_max", "nc_z_width")
_nc_nz = [None]


def _nc_default(p: Dict, k: str) -> float:
    d = {"nc_tau": 0.0, "nc_lnrho_magn": 8.0, "nc_lnrho_width": 2.0,
         "nc_z_max": 10.0 * float(p["dz"]), "nc_z_width": float(p["dz"])}
    return float(p.get(k, d[k]))


def _sync_zgrid(p: Dict) -> None:
    """The vertical grid of this call: p["z"], the positions of the layers
    k = -3 .. nz+2 (strictly increasing), or the uniform z_k = k dz when p
    has none."""
    z = p.get("z")
    if z is None:
        lib().or_set_zgrid(0, None)
        return
    z = np.ascontiguousarray(z, dtype=np.float64)
    if z.shape != (int(p["nz"]) + 2 * NG,) or not np.all(np.diff(z) > 0):
        raise ValueError("p['z'] must hold nz + 6 strictly increasing layer positions")
    lib().or_set_zgrid(int(p["nz"]), _d(z))


def _pvec(p: Dict) -> np.ndarray:
    _sync_zgrid(p)
    if _nc_default(p, "nc_tau") > 0.0 and _nc_nz[0] != int(p["nz"]):
        raise ValueError("Newtonian cooling on: call set_nc_profile(lnrho0, lnT0) for this nz first")
    return np.array([float(p[k]) for k in _PARAM_ORDER] + [_nc_default(p, k) for k in _NC_ORDER],
                    dtype=np.float64)


def set_nc_profile(lnrho0: np.ndarray, lnT0: np.ndarray) -> None:
    """Initial ln rho, ln T profiles ([nz + 6], ghost layers included) that the
    Newtonian cooling term (Sect. 3.1) relaxes toward."""
    lr = np.ascontiguousarray(lnrho0, dtype=np.float64)
    lt = np.ascontiguousarray(lnT0, dtype=np.float64)
    nz = lr.shape[0] - 2 * NG
    lib().or_set_nc_profile(int(nz), _d(lr), _d(lt))
    _nc_nz[0] = nz


def _i(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def to_padded(state: np.ndarray) -> np.ndarray:
    """Interior (8,nz,ny,nx) -> padded state.  The stateful ghost layers of
    u_x, u_y below the photosphere start equal to the photospheric layer."""
    nf, nz, ny, nx = state.shape
    u = np.zeros((nf, nz + 2 * NG, ny + 2 * NG, nx + 2 * NG))
    u[:, NG:NG + nz, NG:NG + ny, NG:NG + nx] = state
    for m in range(1, NG + 1):
        u[3:5, NG - m, NG:NG + ny, NG:NG + nx] = state[3:5, 0]
    return u


def interior(u: np.ndarray) -> np.ndarray:
    return u[:, NG:-NG, NG:-NG, NG:-NG].copy()


def fill_ghosts(p: Dict, u: np.ndarray, lnrho0: np.ndarray, pfe: str = "dft") -> np.ndarray:
    """Fill every ghost cell of the padded state in place (and return it).
    pfe="dft": the potential-field ghosts by the plain DFT (in C);
    pfe="fft": by numpy's FFT (pfe_plane_fft), for large planes."""
    lnrho0 = np.ascontiguousarray(lnrho0, dtype=np.float64)
    if pfe == "dft" or int(p.get("bc_z", 0)) == 1:
        lib().or_fill_ghosts(_i(_dims(p)), _d(_pvec(p)), _d(u), _d(lnrho0))
        return u
    lib().or_fill_ghosts_nopfe(_i(_dims(p)), _d(_pvec(p)), _d(u), _d(lnrho0))
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    lx, ly = nx * p["dx"], ny * p["dy"]
    kt = NG + nz - 1
    if p.get("z") is not None:
        z = np.asarray(p["z"], dtype=np.float64)
        up = [-(z[kt + m] - z[kt]) for m in (1, 2, 3)]
        down = [p["f_pfe_bottom"] * (z[NG] - z[NG - m]) for m in (1, 2, 3)]
    else:
        dz = p["dz"]
        up = [-m * dz for m in (1, 2, 3)]
        down = [p["f_pfe_bottom"] * m * dz for m in (1, 2, 3)]
    for c in range(3):
        top = pfe_plane_fft(lx, ly, u[c, kt, NG:-NG, NG:-NG], up)
        bot = pfe_plane_fft(lx, ly, u[c, NG, NG:-NG, NG:-NG], down)
        for m in (1, 2, 3):
            u[c, kt + m] = np.pad(top[m - 1], NG, mode="wrap")
            u[c, NG - m] = np.pad(bot[m - 1], NG, mode="wrap")
    return u


def a_target(p: Dict, bz: np.ndarray):
    """A_x, A_y of the photospheric target B_z (Sect. 2.4, Eq. 7)."""
    nx, ny = p["nx"], p["ny"]
    bz = np.ascontiguousarray(bz, dtype=np.float64)
    ax = np.zeros((ny, nx))
    ay = np.zeros((ny, nx))
    lib().or_a_target(nx, ny, p["dx"], p["dy"], _d(bz), _d(ax), _d(ay))
    return ax, ay


def a_target_fft(p: Dict, bz: np.ndarray):
    """Same inversion as `a_target` with numpy's FFT as the transform step,
    for planes too large for the plain DFT (pinned against `a_target`)."""
    ny, nx = bz.shape

    def kmod(n, h):
        m = np.arange(n)
        th = 2 * np.pi * np.where(2 * m > n, m - n, m) / n
        k = (45 * np.sin(th) - 9 * np.sin(2 * th) + np.sin(3 * th)) / (30 * h)
        k[(m == 0) | (2 * m == n)] = 0.0
        return k

    kx = kmod(nx, p["dx"])[None, :]
    ky = kmod(ny, p["dy"])[:, None]
    k2 = kx ** 2 + ky ** 2
    bh = np.fft.fft2(bz)
    with np.errstate(divide="ignore", invalid="ignore"):
        ax = np.real(np.fft.ifft2(np.where(k2 > 0, 1j * ky * bh / k2, 0)))
        ay = np.real(np.fft.ifft2(np.where(k2 > 0, -1j * kx * bh / k2, 0)))
    return ax, ay


def rhs(p: Dict, u: np.ndarray, axt, ayt, v0, v1, t0, t1, t) -> np.ndarray:
    """Right-hand side at the cells that carry state (padded array; zero in
    cells that carry none).  `u` must be ghost-filled."""
    out = np.zeros_like(u)
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    lib().or_rhs(_i(_dims(p)), _d(_pvec(p)), _d(u), _d(c(axt)), _d(c(ayt)),
                 _d(c(v0)), _d(c(v1)), t0, t1, t, _d(out))
    return out


def rhs_cells(p: Dict, u: np.ndarray, axt, ayt, v0, v1, t0, t1, t, cells) -> np.ndarray:
    """Right-hand side at the listed interior cells (rows of (k, j, i));
    returns (ncell, 8).  `u` must be ghost-filled."""
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    cl = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((len(cl), 8))
    lib().or_rhs_cells(_i(_dims(p)), _d(_pvec(p)), _d(u), _d(c(axt)), _d(c(ayt)), _d(c(v0)),
                       _d(c(v1)), t0, t1, t, len(cl), _i(cl), _d(out))
    return out


def cfl(p: Dict, u: np.ndarray) -> float:
    return lib().or_cfl(_i(_dims(p)), _d(_pvec(p)), _d(u))


def stats(p: Dict, u: np.ndarray) -> np.ndarray:
    """[E_kin, E_mag, E_th, mass, net flux, unsigned flux, max|div B|]."""
    out = np.zeros(7)
    lib().or_stats(_i(_dims(p)), _d(_pvec(p)), _d(u), _d(out))
    return out


def run(p: Dict, u: np.ndarray, lnrho0, axt, ayt, v0, v1, t0, t1, t, nsteps):
    """Advance the padded state `u` in place by nsteps RK3 steps from time t.
    Returns (t_new, dts)."""
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    tt = np.array([t], dtype=np.float64)
    dts = np.zeros(max(nsteps, 1))
    rc = lib().or_run(_i(_dims(p)), _d(_pvec(p)), _d(u), _d(c(lnrho0)),
                      _d(c(axt)), _d(c(ayt)), _d(c(v0)), _d(c(v1)), t0, t1,
                      _d(tt), int(nsteps), _d(dts))
    if rc != 0:
        raise MemoryError("oracle run failed")
    return float(tt[0]), dts[:nsteps]


def run_case(case, nsteps: Optional[int] = None, params: Optional[Dict] = None):
    """Run a generated case from its initial state; returns (padded u, t, dts)."""
    p = params or case.params
    axt, ayt = a_target(p, case.bz)
    u = to_padded(case.state)
    t, dts = run(p, u, case.lnrho0, axt, ayt, case.v0, case.v1, case.t0,
                 case.t1, 0.0, case.nsteps if nsteps is None else nsteps)
    return u, t, dts


def pfe_plane(nx, ny, lx, ly, plane: np.ndarray, zfacs: Sequence[float]) -> np.ndarray:
    """Potential-field extrapolation of a plane by the plain DFT: returns
    (len(zfacs), ny, nx) with layer o = IDFT(DFT(plane) exp(zfacs[o] |k|))."""
    plane = np.ascontiguousarray(plane, dtype=np.float64)
    z = np.ascontiguousarray(zfacs, dtype=np.float64)
    out = np.zeros((len(z), ny, nx))
    lib().or_pfe_plane(nx, ny, lx, ly, _d(plane), len(z), _d(z), _d(out))
    return out


def pfe_plane_fft(lx, ly, plane: np.ndarray, zfacs: Sequence[float]) -> np.ndarray:
    """Same extrapolation with numpy's FFT as the transform step, for planes
    too large for the plain DFT (pinned against `pfe_plane` at small sizes)."""
    ny, nx = plane.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=lx / nx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=ly / ny)[:, None]
    kk = np.sqrt(kx ** 2 + ky ** 2)
    h = np.fft.fft2(plane)
    return np.stack([np.real(np.fft.ifft2(h * np.exp(zf * kk))) for zf in zfacs])


def deriv(p: Dict, u: np.ndarray, field: int, kind: int, a: int, b: int = 0) -> np.ndarray:
    """Stencil probe: kind 0 = D1 along a, 1 = D2 along a, 2 = D_a D_b."""
    out = np.zeros((p["nz"], p["ny"], p["nx"]))
    lib().or_deriv(_i(_dims(p)), _d(_pvec(p)), _d(u), field, kind, a, b, _d(out))
    return out


def swamp_weight(p: Dict, z: float):
    w = np.zeros(1)
    wp = np.zeros(1)
    lib().or_swamp_weight(_d(_pvec(p)), float(z), _d(w), _d(wp))
    return float(w[0]), float(wp[0])
