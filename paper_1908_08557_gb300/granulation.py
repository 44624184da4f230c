"""The granulation driver (Sect. 2.3, Eqs. 1-4) through libmhd's
mhd_gran_* entry points: argument marshalling only, every step runs in the
CUDA library (there is no CPU fallback).

    gen = Granulation(nx, ny, dx, dy, paper_params(mm_per_unit=0.23))
    gen.update(t, *draws(nx, ny, rng))       # population at time t
    v = gen.velocity(t)                       # [2, ny, nx] driver velocity

Two velocities at times t0 < t1 are the two snapshots mhd_set_driver
interpolates between (the paper's two-step scheme: a 2D granulation run
whose snapshots the 3D model interpolates in time).
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional

import numpy as np

from .binding import MHD_ERR_ARG, MHD_MEM_DEVICE, MHD_MEM_HOST, MHD_OK, GranParams, MHDError, load

# Sect. 2.3's values in Mm, km/s and s
PAPER = dict(r_inner=0.64, r_granule=0.8, r_lane=1.04, v0=1.028, vmin_frac=0.78, lifetime=300.0,
             lifetime_spread=0.10, amp_spread=0.15, f_rot=5.0)


def paper_params(mm_per_unit: float = 1.0, kms_per_unit: float = 1.0, s_per_unit: float = 1.0) -> Dict:
    """Sect. 2.3's parameters in code units, given the code's unit of length
    in Mm, of speed in km/s and of time in s."""
    p = dict(PAPER)
    for k in ("r_inner", "r_granule", "r_lane"):
        p[k] /= mm_per_unit
    p["v0"] /= kms_per_unit
    p["lifetime"] /= s_per_unit
    return p


def draws(nx: int, ny: int, rng: np.random.Generator):
    """One update's random inputs: uint32 visiting keys and two standard
    normal fields (lifetime and amplitude draws), [ny][nx] each."""
    keys = rng.integers(0, 2 ** 32, (ny, nx), dtype=np.uint64).astype(np.uint32)
    return keys, rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))


class Granulation:
    """One mhd_gran generator on a periodic nx x ny plane."""

    def __init__(self, nx: int, ny: int, dx: float, dy: float, params: Optional[Dict] = None,
                 device: str = "cuda:0", stream=None):
        import torch
        self.lib = load()
        self.nx, self.ny = int(nx), int(ny)
        self.device = torch.device(device)
        q = dict(PAPER)
        q.update(params or {})
        self._gp = GranParams(**{k: float(q[k]) for k in PAPER})
        nbytes = int(self.lib.mhd_gran_workspace_bytes(self.nx, self.ny, float(dx), float(dy),
                                                       ctypes.byref(self._gp)))
        if nbytes == 0:
            raise MHDError(MHD_ERR_ARG, "invalid granulation arguments")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.mhd_gran_create(self.nx, self.ny, float(dx), float(dy), ctypes.byref(self._gp),
                                      ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes),
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != MHD_OK:
            raise MHDError(rc, self.lib.mhd_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != MHD_OK:
            raise MHDError(rc, self.lib.mhd_gran_last_error(self.h).decode())

    def _arg(self, a, dtype):
        import torch
        shape = (self.ny, self.nx)
        if isinstance(a, torch.Tensor) and a.is_cuda:
            # keys: 32-bit integers, read as unsigned; draws: float64
            ok = (torch.int32, torch.uint32) if dtype == np.uint32 else (torch.float64,)
            if a.dtype not in ok or tuple(a.shape) != shape or not a.is_contiguous():
                raise ValueError(f"expected a contiguous {shape} tensor of {dtype.__name__}")
            return ctypes.c_void_p(a.data_ptr()), MHD_MEM_DEVICE, a
        arr = np.ascontiguousarray(a if not hasattr(a, "numpy") else a.numpy(), dtype=dtype)
        if arr.shape != shape:
            raise ValueError(f"expected shape {shape}, got {arr.shape}")
        return ctypes.c_void_p(arr.ctypes.data), MHD_MEM_HOST, arr

    def update(self, t: float, keys, c_life, c_amp) -> int:
        """Expire and place granules at time t; returns the parallel rounds."""
        k, mk, a = self._arg(keys, np.uint32)
        cl, ml, b = self._arg(c_life, np.float64)
        ca, ma, c = self._arg(c_amp, np.float64)
        if not (mk == ml == ma):
            raise ValueError("keys, c_life, c_amp must all be host arrays or all device tensors")
        r = ctypes.c_int(0)
        self._check(self.lib.mhd_gran_update(self.h, float(t), k, cl, ca, mk, ctypes.byref(r)))
        del a, b, c
        return int(r.value)

    def velocity(self, t: float, precision: int = 32, out=None):
        """v*_gran at time t as a [2, ny, nx] tensor (float32 or float64)."""
        import torch
        dt = torch.float32 if precision == 32 else torch.float64
        if out is None:
            out = torch.empty((2, self.ny, self.nx), dtype=dt, device=self.device)
        if isinstance(out, np.ndarray):
            self._check(self.lib.mhd_gran_velocity(self.h, float(t), int(precision),
                                                   ctypes.c_void_p(out.ctypes.data), MHD_MEM_HOST))
        else:
            if out.dtype != dt or tuple(out.shape) != (2, self.ny, self.nx) or not out.is_contiguous():
                raise ValueError("out must be a contiguous [2, ny, nx] tensor of the precision's type")
            self._check(self.lib.mhd_gran_velocity(self.h, float(t), int(precision),
                                                   ctypes.c_void_p(out.data_ptr()), MHD_MEM_DEVICE))
        return out

    def granules(self):
        """(occ [ny, nx] int32, par [4, ny, nx] float64: t0, T, v_max, t_max)."""
        import torch
        occ = torch.empty((self.ny, self.nx), dtype=torch.int32, device=self.device)
        par = torch.empty((4, self.ny, self.nx), dtype=torch.float64, device=self.device)
        self._check(self.lib.mhd_gran_read_granules(self.h, ctypes.c_void_p(occ.data_ptr()),
                                                    ctypes.c_void_p(par.data_ptr()), MHD_MEM_DEVICE))
        return occ, par

    def field(self, which: int):
        """Intermediate [2, ny, nx] float64 field of the last velocity():
        0 the granular field, 1 the filtered rotational part (Eq. 3)."""
        import torch
        out = torch.empty((2, self.ny, self.nx), dtype=torch.float64, device=self.device)
        self._check(self.lib.mhd_gran_read_field(self.h, int(which), ctypes.c_void_p(out.data_ptr()),
                                                 MHD_MEM_DEVICE))
        return out

    def launch_count(self) -> int:
        return int(self.lib.mhd_gran_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mhd_gran_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
