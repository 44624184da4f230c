"""Pins of the oracle's Newtonian cooling term (Sect. 3.1, Eqs. 9-10), read
as a relaxation of ln T toward T* = sqrt(T0(z) T'(rho)) at the rate nc_tau,
switched off by a density and a height cut-off with cosine transitions.

Each check isolates the term as the difference of the ln T right-hand side
with the term on and off (everything else in the right-hand side is the
same), on a state with u = 0 and A = 0 in the initial stratification of
`inputs.initial_atmosphere`:
- the initial stratification is a fixed point (T' = T0 at every layer);
- a uniform ln T offset d relaxes at -tau (1 - exp(-d)) below the height
  cut-off, at half that rate at the middle of the cosine step, not at all
  above it;
- the density cut-off passes 1, 0.85, 0.5, 0 at 5, 6.5, 7, 9 e-folds below
  the photospheric density (T' clamped at the top layer there);
- T'(rho) is the piecewise-linear inverse of the initial profile, checked
  against numpy's interpolation of the reversed table.
"""
import math

import numpy as np
import pytest

import inputs
import oracle

NG = oracle.NG
TAU = 0.5


def _box(nz=24, zmax=10.0, zw=3.0):
    p = inputs.scheme_params(8, 8, nz, nc_tau=TAU, nc_z_max=zmax, nc_z_width=zw)
    lt, lr = inputs.initial_atmosphere(nz, p["dz"], p["gz"])
    oracle.set_nc_profile(lr, lt)
    st = np.zeros((8, nz, 8, 8))
    st[6] = lr[NG:NG + nz, None, None]
    st[7] = lt[NG:NG + nz, None, None]
    return p, st, lr, lt


def _term(p, st, lr):
    """The cooling term of each interior cell: ln T right-hand side with the
    term minus without."""
    u = oracle.fill_ghosts(p, oracle.to_padded(st), lr)
    z2, v2 = np.zeros((p["ny"], p["nx"])), np.zeros((2, p["ny"], p["nx"]))
    on = oracle.rhs(p, u, z2, z2, v2, v2, 0.0, 1.0, 0.5)
    off = oracle.rhs(dict(p, nc_tau=0.0), u, z2, z2, v2, v2, 0.0, 1.0, 0.5)
    return oracle.interior(on - off)[7]


def test_initial_stratification_is_a_fixed_point():
    p, st, lr, _ = _box()
    assert np.array_equal(_term(p, st, lr), np.zeros_like(st[7]))


def test_uniform_offset_relaxes_at_tau_below_the_height_cutoff():
    p, st, lr, _ = _box(zmax=10.0, zw=2.0)
    d = 1e-3
    st[7] += d
    got = _term(p, st, lr)[:, 3, 5]
    rate = -TAU * (1.0 - math.exp(-d))
    # z = k dz: full rate up to z_max - w = 8, half at the middle (z = 9),
    # none from z_max = 10 on
    for k in range(0, 9):
        assert got[k] == pytest.approx(rate, rel=1e-12), k
    assert got[9] == pytest.approx(0.5 * rate, rel=1e-12)
    assert np.all(got[10:] == 0.0)
    # relaxation toward T*: cooling for T > T*, heating for T < T*
    st[7] -= 2 * d
    assert np.all(_term(p, st, lr)[:8, 3, 5] > 0.0)


@pytest.mark.parametrize("efolds,cut", [(5.0, 1.0), (6.5, 0.5 * (1 + math.cos(math.pi / 4))), (7.0, 0.5),
                                        (9.0, 0.0)])
def test_density_cutoff(efolds, cut):
    p, st, lr, lt = _box(zmax=100.0, zw=1.0)
    k, d = 4, 1e-4
    L = lr[NG] - efolds
    # T'(rho): the initial ln T where the initial ln rho profile equals L
    # (numpy's interpolation of the reversed table; the top layer beyond it)
    lr_in, lt_in = lr[NG:-NG], lt[NG:-NG]
    lnTp = np.interp(L, lr_in[::-1], lt_in[::-1])
    st[6, k] = L
    st[7, k] = 0.5 * (lt_in[k] + lnTp) + d  # T / T* = e^d
    got = _term(p, st, lr)[k, 4, 4]
    assert got == pytest.approx(-TAU * (1.0 - math.exp(-d)) * cut, rel=1e-9, abs=1e-18)


@pytest.mark.parametrize("frac", [0.0, 0.25, 0.5, 0.9])
def test_inverse_lookup_is_piecewise_linear(frac):
    p, st, lr, lt = _box(zmax=100.0, zw=1.0)
    lr_in, lt_in = lr[NG:-NG], lt[NG:-NG]
    k, m = 2, 9  # the cell at layer 2 takes a density between layers 9 and 10
    L = lr_in[m] + frac * (lr_in[m + 1] - lr_in[m])
    st[6, k] = L
    st[7, k] = lt_in[k]
    # ln T* = (ln T0(z_k) + ln T'(L)) / 2 with ln T' linear in L on the segment
    lnTp = lt_in[m] + frac * (lt_in[m + 1] - lt_in[m])
    r = math.exp(0.5 * (lt_in[k] + lnTp) - lt_in[k])
    cut = 1.0 if lr_in[0] - L <= 6.0 else 0.5 * (1 + math.cos(math.pi * (lr_in[0] - L - 6.0) / 2.0))
    assert _term(p, st, lr)[k, 0, 0] == pytest.approx(-TAU * (1.0 - r) * cut, rel=1e-9)
