"""Manufactured-solution pin of the oracle's full right-hand side.

The continuum right-hand side is built symbolically (SymPy) from the textbook
conservative forms of compressible resistive MHD -- induction u x B - eta
curl B, momentum with grad p / rho and the divergence of the viscous stress
2 rho nu S, continuity d rho/dt = -div(rho u) + D_rho lap rho, internal
energy rho c_v DT/Dt = -p div u + div(kappa0 T^{5/2} grad T) + eta J^2 +
2 rho nu S:S -- plus the swamp terms of Eqs. 18-20 and a constant external
field.  The oracle evaluates the expanded ln-variable forms with sixth-order
stencils; on a smooth triply periodic state its error must fall at sixth
order.  A dropped term, wrong sign or transposed index in the expansion
leaves an O(1) error and fails."""
import numpy as np
import pytest

sp = pytest.importorskip("sympy")

import inputs  # noqa: E402
import oracle  # noqa: E402

NG = oracle.NG

CONST = dict(gamma=5.0 / 3.0, gz=-0.2, nu=0.05, eta=0.04, kappa0=0.03,
             diff_rho=0.06, eta_swamp=0.2, chi_swamp=0.3, diffrho_swamp=0.1,
             z_swamp_start=1.0, z_swamp_end=4.0, bext_x=0.1, bext_y=-0.2,
             bext_z=0.3)


def _symbolic_rhs():
    x, y, z, W, Wp = sp.symbols("x y z W Wp", real=True)
    c = {k: sp.Float(v) for k, v in CONST.items()}
    A = sp.Matrix([0.3 * sp.sin(x + 2 * y) * sp.cos(z) + 0.1 * sp.cos(y),
                   0.2 * sp.cos(x - z) * sp.sin(y),
                   0.25 * sp.sin(x) * sp.cos(y + z)])
    u = sp.Matrix([0.1 * sp.sin(y + z) + 0.05 * sp.cos(x),
                   0.08 * sp.cos(x + z) * sp.sin(y),
                   0.07 * sp.sin(x - y) * sp.cos(z)])
    L = 0.3 * sp.cos(x) * sp.sin(y) + 0.2 * sp.sin(z)
    Th = 0.5 + 0.2 * sp.sin(x + y) * sp.cos(z)
    X = (x, y, z)

    def grad(f):
        return sp.Matrix([f.diff(v) for v in X])

    def div(v):
        return sum(v[i].diff(X[i]) for i in range(3))

    def curl(v):
        return sp.Matrix([v[2].diff(y) - v[1].diff(z), v[0].diff(z) - v[2].diff(x),
                          v[1].diff(x) - v[0].diff(y)])

    def lap(f):
        return sum(f.diff(v, 2) for v in X)

    rho, T = sp.exp(L), sp.exp(Th)
    p = rho * T
    B = curl(A) + sp.Matrix([c["bext_x"], c["bext_y"], c["bext_z"]])
    J = curl(B)
    ez = sp.Matrix([0, 0, 1])
    dA = u.cross(B) - c["eta"] * J + c["eta_swamp"] * W * A.applyfunc(lap) \
        + ez * c["eta_swamp"] * Wp * div(A)
    du_ = sp.Matrix([[u[j].diff(X[i]) for j in range(3)] for i in range(3)])  # d_i u_j
    dv = div(u)
    S = (du_ + du_.T) / 2 - sp.eye(3) * dv / 3
    tau = 2 * rho * c["nu"] * S
    divtau = sp.Matrix([sum(tau[i, j].diff(X[j]) for j in range(3)) for i in range(3)])
    adv = sp.Matrix([sum(u[j] * u[i].diff(X[j]) for j in range(3)) for i in range(3)])
    du = -adv - grad(p) / rho + ez * c["gz"] + J.cross(B) / rho + divtau / rho
    drho = -div(rho * u) + c["diff_rho"] * lap(rho)
    dL = drho / rho + c["diffrho_swamp"] * W * lap(L)
    cv = 1 / (c["gamma"] - 1)
    SS = sum(S[i, j] ** 2 for i in range(3) for j in range(3))
    q = div(c["kappa0"] * T ** sp.Rational(5, 2) * grad(T))
    dT = (-p * dv + q + c["eta"] * J.dot(J) + 2 * rho * c["nu"] * SS) / (rho * cv) \
        - u.dot(grad(T))
    dTh = dT / T + c["chi_swamp"] * W * lap(Th)
    exprs = list(dA) + list(du) + [dL, dTh]
    fields = list(A) + list(u) + [L, Th]
    return (sp.lambdify((x, y, z), fields, "numpy"),
            sp.lambdify((x, y, z, W, Wp), exprs, "numpy"))


def _w(z, zs, zt):
    s = np.clip((z - zs) / (zt - zs), 0.0, 1.0)
    return s * s * (3 - 2 * s), 6 * s * (1 - s) / (zt - zs)


def test_rhs_sixth_order_manufactured():
    fields_f, rhs_f = _symbolic_rhs()
    errs = {}
    for n in (24, 48):
        h = 2 * np.pi / n
        p = inputs.scheme_params(n, n, n, dx=h, dy=h, dz=h, bc_z=1, **CONST)
        cc = np.arange(-NG, n + NG) * h
        Z, Y, X = np.meshgrid(cc, cc, cc, indexing="ij")
        u = np.stack([np.broadcast_to(np.asarray(f, dtype=float), X.shape)
                      for f in fields_f(X, Y, Z)]).copy()
        ci = np.arange(n) * h
        z3, y3, x3 = np.meshgrid(ci, ci, ci, indexing="ij")
        W, Wp = _w(z3, CONST["z_swamp_start"], CONST["z_swamp_end"])
        ex = np.stack([np.broadcast_to(np.asarray(e, dtype=float), x3.shape)
                       for e in rhs_f(x3, y3, z3, W, Wp)])
        got = oracle.interior(oracle.rhs(p, u, np.zeros((n, n)), np.zeros((n, n)),
                                         np.zeros((2, n, n)), np.zeros((2, n, n)),
                                         0.0, 1.0, 0.0))
        errs[n] = np.array([np.abs(got[f] - ex[f]).max() / np.abs(ex[f]).max()
                            for f in range(8)])
    assert np.all(errs[48] < 1e-5), errs[48]
    ratio = errs[24] / errs[48]
    assert np.all(ratio > 40), ratio
