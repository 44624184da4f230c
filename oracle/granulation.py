"""FP64 CPU oracle of the granulation driver (Sect. 2.3, Eqs. 1-4) -- TEST
INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this module; the product never does, and the two share no code.
Plain numpy, written as the section states the method:

* granules live on pixel centres of a periodic nx x ny plane (spacings dx,
  dy); each carries its birth time t0, lifetime T, peak amplitude v_max and
  peak time t_max (Eq. 1);
* an update at time t first removes every granule whose amplitude (Eq. 2)
  has fallen below v_min after its peak, then visits every pixel in the
  order the caller's random keys give (ascending key, then pixel index) and
  starts a granule there when no live centre lies closer than r_inner,
  until the plane is full;
* the velocity at time t superposes the granules' radial fields, amplitude
  Eq. 2 times a radial profile; the rotational part of that field, low-pass
  filtered (Eq. 3), is amplified by f_rot and added back; the sum is scaled
  to the rms speed of the granular field (Eq. 4).

Readings where the section leaves a choice:
the radial profile rises linearly from 0 at the centre to 1 at r_granule
and falls to 0 at r_lane as cos^2; overlapping fields add; T and v_max
take a standard normal draw clipped to [-1, 1] times 10 % and 15 %; the
rotational part is the divergence-free projection, with the mean (k = 0)
and the Nyquist rows and columns carrying none; |k| / k_N is
sqrt((k_x dx / pi)^2 + (k_y dy / pi)^2); the averages of Eq. 4 run over
the plane and both components, and a zero field stays zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class GranParams:
    """Sect. 2.3's values, in the caller's units (lengths as dx, dy)."""
    r_inner: float = 0.64        # no new centre closer to a live one (Mm)
    r_granule: float = 0.8       # granule radius: the radial speed peaks here (Mm)
    r_lane: float = 1.04         # outer edge of the inter-granular lane (Mm)
    v0: float = 1.028            # typical amplitude (km/s)
    vmin_frac: float = 0.78      # v_min / v0
    lifetime: float = 300.0      # T_gran (s)
    lifetime_spread: float = 0.10
    amp_spread: float = 0.15
    f_rot: float = 5.0


def t_max(T, v_max, v_min):
    """Eq. 1: the time after birth at which the amplitude peaks."""
    return T * math.sqrt(abs(math.log(v_min / v_max)))


def amplitude(t, t0, T, v_max, tm):
    """Eq. 2: the life cycle of a granule's amplitude."""
    return v_max * math.exp(-((t - t0 - tm) / T) ** 2)


class Granulation:
    """The granules of a periodic plane, one possible per pixel (a dict from
    pixel (j, i) to (t0, T, v_max, t_max))."""

    def __init__(self, nx, ny, dx, dy, gp: GranParams):
        self.nx, self.ny, self.dx, self.dy, self.gp = nx, ny, dx, dy, gp
        self.live = {}

    def _dist2(self, j0, i0, j1, i1):
        """Squared distance of pixel centres (j0, i0) and (j1, i1) (arrays),
        nearest periodic image."""
        di = (i1 - i0) % self.nx
        dj = (j1 - j0) % self.ny
        di = np.minimum(di, self.nx - di)
        dj = np.minimum(dj, self.ny - dj)
        return (di * self.dx) ** 2 + (dj * self.dy) ** 2

    def expire(self, t):
        """Remove granules whose amplitude has dropped below v_min after
        the peak: t - t0 - t_max > t_max (Eq. 2 equals v_min at
        t0 + 2 t_max, by Eq. 1)."""
        for key, (t0, T, vm, tm) in list(self.live.items()):
            if t - t0 - tm > tm:
                del self.live[key]

    def place(self, t, keys, g_life, g_amp):
        """Fill the plane: visit the pixels by ascending (key, index) and start
        a granule at each one with no live centre closer than r_inner.  keys,
        g_life, g_amp: [ny][nx] random draws (uint32 keys, standard normals)."""
        gp = self.gp
        v_min = gp.vmin_frac * gp.v0
        order = sorted(range(self.nx * self.ny), key=lambda q: (int(keys.flat[q]), q))
        r2 = gp.r_inner ** 2
        cj = np.array([c[0] for c in self.live], dtype=np.int64)
        ci = np.array([c[1] for c in self.live], dtype=np.int64)
        for q in order:
            j, i = divmod(q, self.nx)
            if cj.size and np.min(self._dist2(j, i, cj, ci)) < r2:
                continue
            cl = min(1.0, max(-1.0, float(g_life.flat[q])))
            ca = min(1.0, max(-1.0, float(g_amp.flat[q])))
            T = gp.lifetime * (1.0 + gp.lifetime_spread * cl)
            vm = gp.v0 * (1.0 + gp.amp_spread * ca)
            self.live[(j, i)] = (t, T, vm, t_max(T, vm, v_min))
            cj = np.append(cj, j)
            ci = np.append(ci, i)

    def update(self, t, keys, g_life, g_amp):
        self.expire(t)
        self.place(t, keys, g_life, g_amp)

    def maps(self):
        """Pixel maps: occupancy (int32) and t0, T, v_max, t_max (float64)."""
        occ = np.zeros((self.ny, self.nx), np.int32)
        par = np.zeros((4, self.ny, self.nx))
        for (j, i), v in self.live.items():
            occ[j, i] = 1
            par[:, j, i] = v
        return occ, par

    def granular_field(self, t):
        """v_gran: every live granule adds amplitude (Eq. 2) x profile(r) x
        the unit vector away from its centre, r the nearest-image distance."""
        gp = self.gp
        x = np.arange(self.nx)[None, :]
        y = np.arange(self.ny)[:, None]
        vx = np.zeros((self.ny, self.nx))
        vy = np.zeros((self.ny, self.nx))
        for (cj, ci), (t0, T, vm, tm) in self.live.items():
            a = amplitude(t, t0, T, vm, tm)
            ox = ((x - ci + self.nx // 2) % self.nx - self.nx // 2) * self.dx
            oy = ((y - cj + self.ny // 2) % self.ny - self.ny // 2) * self.dy
            ox, oy = np.broadcast_arrays(ox, oy)
            r = np.hypot(ox, oy)
            prof = radial_profile(r, gp.r_granule, gp.r_lane)
            with np.errstate(invalid="ignore", divide="ignore"):
                ux = np.where(r > 0, ox / r, 0.0)
                uy = np.where(r > 0, oy / r, 0.0)
            vx += a * prof * ux
            vy += a * prof * uy
        return vx, vy

    def granular_field_at(self, t, pix):
        """v_gran at the pixels pix [(j, i), ...] only: the sum over every live
        granule, one pixel at a time (for planes too large for the full map)."""
        gp = self.gp
        c = np.array(list(self.live.keys()), dtype=np.int64).reshape(-1, 2)
        par = np.array(list(self.live.values()), dtype=np.float64).reshape(-1, 4)
        a = par[:, 2] * np.exp(-((t - par[:, 0] - par[:, 3]) / par[:, 1]) ** 2)
        out = np.zeros((len(pix), 2))
        for n, (j, i) in enumerate(pix):
            ox = ((i - c[:, 1] + self.nx // 2) % self.nx - self.nx // 2) * self.dx
            oy = ((j - c[:, 0] + self.ny // 2) % self.ny - self.ny // 2) * self.dy
            r = np.hypot(ox, oy)
            near = (r > 0) & (r < gp.r_lane)
            f = a[near] * radial_profile(r[near], gp.r_granule, gp.r_lane) / r[near]
            out[n] = (np.sum(f * ox[near]), np.sum(f * oy[near]))
        return out

    def velocity(self, t):
        """v*_gran (Eq. 4) at time t, with the filtered rotational part."""
        vx, vy = self.granular_field(t)
        rx, ry = rotational_part(vx, vy, self.dx, self.dy)
        wx = vx + self.gp.f_rot * rx
        wy = vy + self.gp.f_rot * ry
        return renormalise(vx, vy, wx, wy)


def radial_profile(r, r_g, r_l):
    """Radial speed / amplitude at distance r from the centre: r / r_g up to
    r_g, cos^2 down to 0 at r_l, 0 beyond."""
    r = np.asarray(r, dtype=np.float64)
    rise = r / r_g
    fall = np.cos(0.5 * np.pi * (r - r_g) / (r_l - r_g)) ** 2
    return np.where(r <= r_g, rise, np.where(r < r_l, fall, 0.0))


def rotational_part(vx, vy, dx, dy):
    """Eq. 3: the divergence-free part of (vx, vy) (projection
    v - k (k . v) / |k|^2 of the 2D FFT), times exp(-(2 |k| / k_N)^4), back in
    real space; the mean and the Nyquist rows and columns dropped."""
    ny, nx = vx.shape
    fx = np.fft.fft2(vx)
    fy = np.fft.fft2(vy)
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=dx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=dy)[:, None]
    kx, ky = np.broadcast_arrays(kx, ky)
    k2 = kx ** 2 + ky ** 2
    keep = k2 > 0
    if nx % 2 == 0:
        keep &= np.arange(nx)[None, :] != nx // 2
    if ny % 2 == 0:
        keep &= np.arange(ny)[:, None] != ny // 2
    safe = np.where(keep, k2, 1.0)
    div = (kx * fx + ky * fy) / safe
    px = np.where(keep, fx - kx * div, 0.0)
    py = np.where(keep, fy - ky * div, 0.0)
    kn2 = (kx * dx / np.pi) ** 2 + (ky * dy / np.pi) ** 2
    w = np.exp(-(4.0 * kn2) ** 2)       # (2 |k| / k_N)^4
    return np.fft.ifft2(w * px).real, np.fft.ifft2(w * py).real


def renormalise(vx, vy, wx, wy):
    """Eq. 4: scale (wx, wy) to the rms speed of (vx, vy)."""
    sv = float(np.sum(vx * vx + vy * vy))
    sw = float(np.sum(wx * wx + wy * wy))
    if sw == 0.0:
        return np.zeros_like(wx), np.zeros_like(wy)
    s = math.sqrt(sv / sw)
    return wx * s, wy * s
