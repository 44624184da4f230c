"""Pins of the oracle on a non-uniform vertical grid (the production grid's
spacing grows from about 100 km to about 800 km, Sect. 1; the ghost rules
of Sects. 2.5 and 4.1 and Eq. 17 written with the layer positions):
- the chain rule: D_z z = 1, D_z^2 z = 0, D_x D_z (x z) = 1;
- the full right-hand side against the manufactured solution on a
  stretched, triply periodic grid falls at sixth order;
- an isothermal hydrostatic column on a stretched grid is a fixed point of
  the bottom (Eq. 8) and top (Eq. 13) ghost rules;
- one Fourier mode of A is extrapolated over z_{nz-1+m} - z_{nz-1} upward
  (Eq. 17) and f_b (z_0 - z_{-m}) downward;
- the CFL step takes the local spacing; cell volumes are the cells'
  vertical extents (z_{k+1} - z_{k-1}) / 2; div B stays zero;
- positions k dz given explicitly reproduce the uniform grid.
"""
import math

import numpy as np
import pytest

import inputs
import oracle

NG = oracle.NG


def _periodic_z(n, L, a):
    """z(xi) = L (xi / n + a sin(2 pi xi / n) / (2 pi)) at xi = -3 .. n+2:
    z(xi + n) = z(xi) + L, so the periodic copies of the fields sit at
    their periodic positions; z'(xi) = (L / n)(1 + a cos(2 pi xi / n))."""
    k = np.arange(-NG, n + NG, dtype=np.float64)
    return L * (k / n + a * np.sin(2 * np.pi * k / n) / (2 * np.pi))


def _padded_from(fn, p, z):
    """Padded array of fn(x, y, z) (every field the same function)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x = np.arange(-NG, nx + NG) * p["dx"]
    y = np.arange(-NG, ny + NG) * p["dy"]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    one = fn(X, Y, Z)
    return np.ascontiguousarray(np.broadcast_to(one, (8,) + one.shape))


def test_chain_rule_identities():
    z, _, _ = inputs.stretched_z(24, 0.3, 1.7, 12, 4)
    p = dict(inputs.scheme_params(8, 8, 24, dx=0.5, dy=0.7, dz=1.0), z=z)
    u = _padded_from(lambda X, Y, Z: Z, p, z)
    assert np.max(np.abs(oracle.deriv(p, u, 6, 0, 2) - 1.0)) < 1e-12
    assert np.max(np.abs(oracle.deriv(p, u, 6, 1, 2))) < 1e-11
    u = _padded_from(lambda X, Y, Z: X * Z, p, z)
    assert np.max(np.abs(oracle.deriv(p, u, 6, 2, 0, 2) - 1.0)) < 1e-11
    assert np.max(np.abs(oracle.deriv(p, u, 6, 2, 2, 0) - 1.0)) < 1e-11


def test_rhs_sixth_order_on_a_stretched_grid():
    from test_oracle_mms import CONST, _symbolic_rhs, _w
    fields_f, rhs_f = _symbolic_rhs()
    errs = {}
    for n in (24, 48):
        h = 2 * np.pi / n
        z = _periodic_z(n, 2 * np.pi, 0.3)
        p = dict(inputs.scheme_params(n, n, n, dx=h, dy=h, dz=h, bc_z=1, **CONST), z=z)
        cc = np.arange(-NG, n + NG) * h
        Z, Y, X = np.meshgrid(z, cc, cc, indexing="ij")
        u = np.stack([np.broadcast_to(np.asarray(f, dtype=float), X.shape)
                      for f in fields_f(X, Y, Z)]).copy()
        ci = np.arange(n) * h
        z3, y3, x3 = np.meshgrid(z[NG:-NG], ci, ci, indexing="ij")
        W, Wp = _w(z3, CONST["z_swamp_start"], CONST["z_swamp_end"])
        ex = np.stack([np.broadcast_to(np.asarray(e, dtype=float), x3.shape)
                       for e in rhs_f(x3, y3, z3, W, Wp)])
        got = oracle.interior(oracle.rhs(p, u, np.zeros((n, n)), np.zeros((n, n)),
                                         np.zeros((2, n, n)), np.zeros((2, n, n)), 0.0, 1.0, 0.0))
        errs[n] = np.array([np.abs(got[f] - ex[f]).max() / np.abs(ex[f]).max() for f in range(8)])
    assert np.all(errs[48] < 1e-4), errs[48]
    ratio = errs[24] / errs[48]
    assert np.all(ratio > 40), ratio


def _column(nz=20, T=1.3):
    z, _, _ = inputs.stretched_z(nz, 0.25, 2.0, nz / 2, 3)
    # the nominal dz differs from the spacing at both ends on purpose
    p = dict(inputs.scheme_params(8, 8, nz, dz=1.0), z=z)
    lnrho = p["gz"] * z / T
    st = np.zeros((8, nz, 8, 8))
    st[6] = lnrho[NG:-NG, None, None]
    st[7] = math.log(T)
    return p, z, lnrho, oracle.to_padded(st)


def test_isothermal_column_is_a_fixed_point():
    T = 1.3
    p, z, lnrho, u = _column(T=T)
    oracle.fill_ghosts(p, u, lnrho)
    nz = p["nz"]
    for m in range(1, NG + 1):
        # bottom: ln T from Eq. 8 with the local spacing z_{j+1} - z_j
        assert np.allclose(u[7, NG - m], math.log(T), rtol=0, atol=1e-14)
        # top: ln rho from Eq. 13 over z_{nz-1+m} - z_{nz-1-m}
        assert np.allclose(u[6, NG + nz - 1 + m], lnrho[NG + nz - 1 + m], rtol=0, atol=1e-13)
        assert np.allclose(u[7, NG + nz - 1 + m], math.log(T), rtol=0, atol=0)


def test_potential_field_mode_over_layer_distances():
    p, z, lnrho, u = _column()
    nx = ny = 8
    kx = 2 * np.pi * 2 / (nx * p["dx"])
    x = np.arange(-NG, nx + NG) * p["dx"]
    nz = p["nz"]
    kt = NG + nz - 1
    u[0, kt] = np.cos(kx * x)[None, :]
    u[0, NG] = np.cos(kx * x)[None, :]
    oracle.fill_ghosts(p, u, lnrho)
    for m in range(1, NG + 1):
        up = np.cos(kx * x) * math.exp(-kx * (z[kt + m] - z[kt]))
        down = np.cos(kx * x) * math.exp(p["f_pfe_bottom"] * kx * (z[NG] - z[NG - m]))
        assert np.allclose(u[0, kt + m], up[None, :], rtol=0, atol=1e-13)
        assert np.allclose(u[0, NG - m], down[None, :], rtol=0, atol=1e-13)


def test_cfl_takes_the_local_spacing():
    nz = 24
    z, zp, _ = inputs.stretched_z(nz, 0.3, 1.7, 12, 4)
    # no swamp layer: the diffusive limit is the bulk diffusivity alone
    p = dict(inputs.scheme_params(8, 8, nz, dx=2.0, dy=2.0, dz=1.0, eta_swamp=0.0, chi_swamp=0.0,
                                  diffrho_swamp=0.0), z=z)
    st = np.zeros((8, nz, 8, 8))
    st[5] = 0.05  # u_z
    u = oracle.fill_ghosts(p, oracle.to_padded(st), np.zeros(nz + 2 * NG))
    got = oracle.cfl(p, u)
    # the finest layer (the bottom one, z' = 0.3 to 6th order) sets both limits
    inv2 = 2 / 4.0 + 1 / zp[NG:-NG] ** 2
    adv = np.max(0.05 / zp[NG:-NG] + math.sqrt(p["gamma"]) * np.sqrt(inv2))
    dmax = max(p["nu"], p["eta"], p["diff_rho"], (p["gamma"] - 1) * p["kappa0"])
    want = min(p["c_adv"] / adv, p["c_diff"] / (dmax * np.max(inv2)))
    assert got == pytest.approx(want, rel=1e-5)


def test_cell_volumes_and_div_b():
    nz = 16
    z, _, _ = inputs.stretched_z(nz, 0.3, 1.7, 8, 3)
    p = dict(inputs.scheme_params(8, 8, nz, dx=0.5, dy=0.75, dz=1.0), z=z)
    rng = np.random.default_rng(2)
    st = np.zeros((8, nz, 8, 8))
    st[0:3] = 0.1 * rng.standard_normal((3, nz, 8, 8))
    u = oracle.fill_ghosts(p, oracle.to_padded(st), np.zeros(nz + 2 * NG))
    s = oracle.stats(p, u)
    # rho = T = 1: mass = dx dy nx ny sum_k (z_{k+1} - z_{k-1}) / 2, which
    # telescopes to (z_nz + z_{nz-1} - z_0 - z_{-1}) / 2
    vol = 0.5 * 0.75 * 64 * 0.5 * (z[NG + nz] + z[NG + nz - 1] - z[NG] - z[NG - 1])
    # stats: [E_kin, E_mag, E_th, mass, net flux, unsigned flux, max |div B|]
    assert s[3] == pytest.approx(vol, rel=1e-13)
    assert s[2] == pytest.approx(vol / (p["gamma"] - 1), rel=1e-13)
    assert s[6] < 1e-12


def test_uniform_positions_reproduce_the_uniform_grid():
    case = inputs.make_box(16, 16, 12, seed=4, magnetogram="bipoles", n_mag=4)
    p = case.params
    pz = dict(p, z=np.arange(-NG, p["nz"] + NG) * p["dz"])
    rng = np.random.default_rng(1)
    st = case.state.copy()
    st[3:6] += 0.02 * rng.standard_normal(st[3:6].shape)
    axt, ayt = oracle.a_target(p, case.bz)
    outs = []
    for q in (p, pz):
        u = oracle.fill_ghosts(q, oracle.to_padded(st), case.lnrho0)
        r = oracle.rhs(q, u, axt, ayt, case.v0, case.v1, case.t0, case.t1, 0.3)
        outs.append((u, r, oracle.cfl(q, u), oracle.stats(q, u)))
    (u0, r0, c0, s0), (u1, r1, c1, s1) = outs
    assert np.allclose(u1, u0, rtol=1e-13, atol=1e-13)
    for f in range(8):
        sc = np.abs(r0[f]).max()
        assert np.max(np.abs(r1[f] - r0[f])) <= 1e-11 * sc, f
    assert c1 == pytest.approx(c0, rel=1e-13)
    for k in range(4):  # E_kin, E_mag, E_th, mass
        assert s1[k] == pytest.approx(s0[k], rel=1e-13)
