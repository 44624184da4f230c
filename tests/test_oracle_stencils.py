"""Pins of the oracle's sixth-order stencils (first, second, mixed):
exact on polynomials of degree <= 6, sixth-order convergence on periodic
sine fields (error ratio -> 2^6 = 64 under grid halving)."""
import numpy as np
import pytest

import oracle

NG = oracle.NG


def _box(n, h, **over):
    p = dict(nx=n, ny=n, nz=n, bc_z=1, dx=h, dy=h, dz=h, gamma=5 / 3, gz=0.0,
             nu=0.0, eta=0.0, kappa0=0.0, diff_rho=0.0, eta_swamp=0.0,
             chi_swamp=0.0, diffrho_swamp=0.0, z_swamp_start=0.0,
             z_swamp_end=0.0, tau_u=0.0, tau_A=0.0, t_ramp=0.0,
             f_pfe_bottom=0.2, c_adv=0.4, c_diff=0.25, dt_fixed=0.0,
             bext_x=0.0, bext_y=0.0, bext_z=0.0)
    p.update(over)
    return p


def _coords(n, h):
    c = (np.arange(-NG, n + NG)) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z


@pytest.mark.parametrize("deg", [1, 2, 3, 4, 5, 6])
def test_exact_on_polynomials(deg):
    n, h = 10, 0.37
    p = _box(n, h)
    x, y, z = _coords(n, h)
    # f = x^deg + 0.5 y^deg - 0.3 z^deg + x^a y^b z^c cross terms of total deg
    a = deg // 2
    f = x ** deg + 0.5 * y ** deg - 0.3 * z ** deg + 0.7 * x ** a * y ** (deg - a) \
        + 0.2 * y ** a * z ** (deg - a) - 0.4 * z ** a * x ** (deg - a)
    u = np.zeros((8,) + f.shape)
    u[0] = f
    sl = (slice(NG, -NG),) * 3
    X, Y, Z = x[sl], y[sl], z[sl]

    def ex_d1(axis):
        if axis == 0:
            return deg * X ** (deg - 1) + 0.7 * a * X ** max(a - 1, 0) * Y ** (deg - a) * (a > 0) \
                - 0.4 * (deg - a) * Z ** a * X ** max(deg - a - 1, 0) * (deg - a > 0)
        if axis == 1:
            return 0.5 * deg * Y ** (deg - 1) + 0.7 * (deg - a) * X ** a * Y ** max(deg - a - 1, 0) * (deg - a > 0) \
                + 0.2 * a * Y ** max(a - 1, 0) * Z ** (deg - a) * (a > 0)
        return -0.3 * deg * Z ** (deg - 1) + 0.2 * (deg - a) * Y ** a * Z ** max(deg - a - 1, 0) * (deg - a > 0) \
            - 0.4 * a * Z ** max(a - 1, 0) * X ** (deg - a) * (a > 0)

    scale = np.abs(f).max()
    for axis in range(3):
        got = oracle.deriv(p, u, 0, 0, axis)
        assert np.allclose(got, ex_d1(axis), rtol=0, atol=1e-11 * scale / h), axis
    # second derivatives along each axis of the pure powers
    if deg >= 2:
        ex = [deg * (deg - 1) * X ** (deg - 2), 0.5 * deg * (deg - 1) * Y ** (deg - 2),
              -0.3 * deg * (deg - 1) * Z ** (deg - 2)]
        g = np.zeros((8,) + f.shape)
        for axis, coord, c in ((0, x, 1.0), (1, y, 0.5), (2, z, -0.3)):
            g[0] = c * coord ** deg
            got = oracle.deriv(p, g, 0, 1, axis)
            assert np.allclose(got, ex[axis], rtol=0, atol=1e-10 * scale / h ** 2), axis
    # mixed derivative of x^a y^b (a + b = deg): a b x^(a-1) y^(b-1)
    for (aa, bb) in [(a, deg - a), (deg - a, a)]:
        if aa == 0 or bb == 0:
            continue
        g = np.zeros((8,) + f.shape)
        g[0] = x ** aa * y ** bb
        got = oracle.deriv(p, g, 0, 2, 0, 1)
        exm = aa * bb * X ** (aa - 1) * Y ** (bb - 1)
        assert np.allclose(got, exm, rtol=0, atol=1e-10 * scale / h ** 2)
        got = oracle.deriv(p, g, 0, 2, 1, 0)
        assert np.allclose(got, exm, rtol=0, atol=1e-10 * scale / h ** 2)


def test_sixth_order_convergence():
    errs = {}
    for n in (16, 32):
        h = 2 * np.pi / n
        p = _box(n, h)
        x, y, z = _coords(n, h)
        u = np.zeros((8,) + x.shape)
        u[0] = np.sin(x + 0.3) * np.cos(2 * y) * np.sin(z - 0.1)
        sl = (slice(NG, -NG),) * 3
        X, Y, Z = x[sl], y[sl], z[sl]
        e = []
        e.append(np.abs(oracle.deriv(p, u, 0, 0, 0) - np.cos(X + 0.3) * np.cos(2 * Y) * np.sin(Z - 0.1)).max())
        e.append(np.abs(oracle.deriv(p, u, 0, 0, 1) + 2 * np.sin(X + 0.3) * np.sin(2 * Y) * np.sin(Z - 0.1)).max())
        e.append(np.abs(oracle.deriv(p, u, 0, 1, 1) + 4 * np.sin(X + 0.3) * np.cos(2 * Y) * np.sin(Z - 0.1)).max())
        e.append(np.abs(oracle.deriv(p, u, 0, 1, 2) + np.sin(X + 0.3) * np.cos(2 * Y) * np.sin(Z - 0.1)).max())
        e.append(np.abs(oracle.deriv(p, u, 0, 2, 0, 2) - np.cos(X + 0.3) * np.cos(2 * Y) * np.cos(Z - 0.1)).max())
        e.append(np.abs(oracle.deriv(p, u, 0, 2, 1, 2) + 2 * np.sin(X + 0.3) * np.sin(2 * Y) * np.cos(Z - 0.1)).max())
        errs[n] = np.array(e)
    ratio = errs[16] / errs[32]
    assert np.all(ratio > 50) and np.all(ratio < 80), ratio
