"""Thin ctypes binding of libmhd (include/mhd.h): argument marshalling only.

Every step of the method runs inside the CUDA library; this module converts
Python arguments (torch tensors on the GPU, or numpy arrays on the host) into
the pointers, sizes and flags of the C ABI.  Device memory (the one
workspace) comes from PyTorch's allocator; the library itself allocates none.
There is no CPU fallback: if libmhd.so is missing or cannot be loaded, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhd.so")

MHD_OK = 0
MHD_ERR_ARG = -1
MHD_ERR_WORKSPACE = -2
MHD_ERR_CUDA = -3
MHD_ERR_NONFINITE = -4
MHD_ERR_UNSUPPORTED = -5
MHD_ERR_TIMEOUT = -6
MHD_ERR_IO = -7
MHD_MEM_DEVICE = 0
MHD_MEM_HOST = 1
NFIELD = 8
NGHOST = 3

EXPORTED = ("mhd_workspace_bytes", "mhd_create", "mhd_set_driver", "mhd_step",
            "mhd_read", "mhd_write", "mhd_read_stats", "mhd_get_time",
            "mhd_destroy", "mhd_last_error", "mhd_fill_ghosts",
            "mhd_read_padded", "mhd_eval_rhs", "mhd_compute_dt",
            "mhd_compute_stats", "mhd_read_target", "mhd_profile",
            "mhd_read_profile", "mhd_launch_count", "mhd_invert_magnetogram_static",
            "mhd_set_time", "mhd_checkpoint_bytes", "mhd_save", "mhd_restore",
            "mhd_adjoint_init", "mhd_adjoint_step", "mhd_adjoint_read", "mhd_bz_plane",
            "mhd_bz_plane_adjoint", "mhd_gran_workspace_bytes", "mhd_gran_create", "mhd_gran_update",
            "mhd_gran_velocity", "mhd_gran_read_granules", "mhd_gran_read_field", "mhd_gran_launch_count",
            "mhd_gran_last_error", "mhd_gran_destroy", "mhd_set_a_background",
            "mhd_debug_skip_copy", "mhd_read_plane", "mhd_fma_peak", "mhd_tape_bytes", "mhd_step_taped",
            "mhd_adjoint_step_taped", "mhd_write_snapshot", "mhd_h5_write", "mhd_h5_checksum")
KERNEL_CLASSES = ("ghost", "pfe", "cfl", "stats", "rk")


class MHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmhd error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("precision", ctypes.c_int), ("bc_z", ctypes.c_int),
                ("stats_every", ctypes.c_int), ("adjoint", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("gamma", ctypes.c_double), ("gz", ctypes.c_double),
                ("nu", ctypes.c_double), ("eta", ctypes.c_double),
                ("kappa0", ctypes.c_double), ("diff_rho", ctypes.c_double),
                ("eta_swamp", ctypes.c_double), ("chi_swamp", ctypes.c_double),
                ("diffrho_swamp", ctypes.c_double),
                ("z_swamp_start", ctypes.c_double), ("z_swamp_end", ctypes.c_double),
                ("tau_u", ctypes.c_double), ("tau_A", ctypes.c_double),
                ("t_ramp", ctypes.c_double), ("f_pfe_bottom", ctypes.c_double),
                ("c_adv", ctypes.c_double), ("c_diff", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("bext", ctypes.c_double * 3),
                ("nc_tau", ctypes.c_double), ("nc_lnrho_magn", ctypes.c_double),
                ("nc_lnrho_width", ctypes.c_double), ("nc_z_max", ctypes.c_double),
                ("nc_z_width", ctypes.c_double), ("a_background", ctypes.c_int),
                ("z", ctypes.POINTER(ctypes.c_double))]


class Stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("e_kin", ctypes.c_double), ("e_mag", ctypes.c_double),
                ("e_th", ctypes.c_double), ("mass", ctypes.c_double),
                ("flux_net", ctypes.c_double), ("flux_abs", ctypes.c_double),
                ("divb_max", ctypes.c_double), ("step", ctypes.c_longlong),
                ("nonfinite", ctypes.c_int), ("pad_", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class GranParams(ctypes.Structure):
    """mhd_gran_params (Sect. 2.3): lengths in the units of dx, dy."""
    _fields_ = [(n, ctypes.c_double) for n in ("r_inner", "r_granule", "r_lane", "v0", "vmin_frac", "lifetime",
                                               "lifetime_spread", "amp_spread", "f_rot")]


_lib = None


def load(path: Optional[str] = None):
    """Load libmhd.so (build it first with paper_1908_08557_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libmhd.so not found at {p}: run __graft_entry__.build() "
                           "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(p)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER(Params)
    lib.mhd_workspace_bytes.argtypes = [P]
    lib.mhd_workspace_bytes.restype = sz
    dpp = ctypes.POINTER(ctypes.c_double)
    lib.mhd_create.argtypes = [P, vp, sz, vp, i, dpp, dpp, vp, ctypes.POINTER(vp)]
    lib.mhd_set_driver.argtypes = [vp, vp, vp, vp, d, d, i]
    lib.mhd_set_a_background.argtypes = [vp, vp, vp, i]
    lib.mhd_debug_skip_copy.argtypes = [vp, i, i]
    lib.mhd_read_plane.argtypes = [vp, i, i, vp, i]
    lib.mhd_fma_peak.argtypes = [i, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.mhd_write_snapshot.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
    lib.mhd_h5_write.argtypes = [ctypes.c_char_p, ctypes.c_char_p, P, d, vp]
    lib.mhd_h5_checksum.argtypes = [vp, sz]
    lib.mhd_h5_checksum.restype = ctypes.c_uint
    lib.mhd_tape_bytes.argtypes = [vp]
    lib.mhd_tape_bytes.restype = sz
    lib.mhd_step_taped.argtypes = [vp, vp]
    lib.mhd_adjoint_step_taped.argtypes = [vp, vp]
    lib.mhd_step.argtypes = [vp, i]
    lib.mhd_read.argtypes = [vp, i, vp, i]
    lib.mhd_write.argtypes = [vp, vp, i]
    lib.mhd_read_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.mhd_get_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mhd_destroy.argtypes = [vp]
    lib.mhd_destroy.restype = None
    lib.mhd_last_error.argtypes = [vp]
    lib.mhd_last_error.restype = ctypes.c_char_p
    lib.mhd_fill_ghosts.argtypes = [vp]
    lib.mhd_read_padded.argtypes = [vp, i, vp, i]
    lib.mhd_eval_rhs.argtypes = [vp, d, vp, i]
    lib.mhd_compute_dt.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.mhd_compute_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.mhd_read_target.argtypes = [vp, vp, i]
    lib.mhd_profile.argtypes = [vp, i]
    lib.mhd_read_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_longlong)]
    lib.mhd_invert_magnetogram_static.argtypes = [i, i, d, d, i, vp, vp, vp, vp]
    lib.mhd_set_time.argtypes = [vp, d]
    lib.mhd_checkpoint_bytes.argtypes = [vp]
    lib.mhd_checkpoint_bytes.restype = sz
    lib.mhd_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.mhd_restore.argtypes = [vp, vp, d]
    lib.mhd_adjoint_init.argtypes = [vp, vp, i]
    lib.mhd_adjoint_step.argtypes = [vp]
    lib.mhd_adjoint_read.argtypes = [vp, vp, vp, vp, vp, i]
    lib.mhd_bz_plane.argtypes = [vp, vp, i, vp]
    lib.mhd_bz_plane_adjoint.argtypes = [vp, vp, i, vp]
    lib.mhd_launch_count.argtypes = [vp]
    lib.mhd_launch_count.restype = ctypes.c_longlong
    G = ctypes.POINTER(GranParams)
    lib.mhd_gran_workspace_bytes.argtypes = [i, i, d, d, G]
    lib.mhd_gran_workspace_bytes.restype = sz
    lib.mhd_gran_create.argtypes = [i, i, d, d, G, vp, sz, vp, ctypes.POINTER(vp)]
    lib.mhd_gran_update.argtypes = [vp, d, vp, vp, vp, i, ctypes.POINTER(ctypes.c_int)]
    lib.mhd_gran_velocity.argtypes = [vp, d, i, vp, i]
    lib.mhd_gran_read_granules.argtypes = [vp, vp, vp, i]
    lib.mhd_gran_read_field.argtypes = [vp, i, vp, i]
    lib.mhd_gran_launch_count.argtypes = [vp]
    lib.mhd_gran_launch_count.restype = ctypes.c_longlong
    lib.mhd_gran_last_error.argtypes = [vp]
    lib.mhd_gran_last_error.restype = ctypes.c_char_p
    lib.mhd_gran_destroy.argtypes = [vp]
    lib.mhd_gran_destroy.restype = None
    for name in EXPORTED:
        if name not in ("mhd_workspace_bytes", "mhd_destroy", "mhd_last_error", "mhd_tape_bytes", "mhd_h5_checksum",
                        "mhd_launch_count", "mhd_checkpoint_bytes", "mhd_gran_workspace_bytes",
                        "mhd_gran_launch_count", "mhd_gran_last_error", "mhd_gran_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def make_params(p: Dict, precision: int = 32, stats_every: int = 0, adjoint: bool = False,
                a_background: bool = False) -> Params:
    q = Params()
    q.nx, q.ny, q.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])
    q.precision = int(precision)
    q.bc_z = int(p.get("bc_z", 0))
    q.stats_every = int(stats_every)
    q.adjoint = 1 if adjoint else 0
    for k in ("dx", "dy", "dz", "gamma", "gz", "nu", "eta", "kappa0", "diff_rho",
              "eta_swamp", "chi_swamp", "diffrho_swamp", "z_swamp_start",
              "z_swamp_end", "tau_u", "tau_A", "t_ramp", "f_pfe_bottom", "c_adv",
              "c_diff", "dt_fixed"):
        setattr(q, k, float(p[k]))
    q.bext[0], q.bext[1], q.bext[2] = (float(p.get("bext_x", 0.0)),
                                       float(p.get("bext_y", 0.0)),
                                       float(p.get("bext_z", 0.0)))
    # Newtonian cooling: off unless nc_tau > 0
    q.nc_tau = float(p.get("nc_tau", 0.0))
    q.nc_lnrho_magn = float(p.get("nc_lnrho_magn", 8.0))
    q.nc_lnrho_width = float(p.get("nc_lnrho_width", 2.0))
    q.nc_z_max = float(p.get("nc_z_max", 10.0 * float(p["dz"])))
    q.nc_z_width = float(p.get("nc_z_width", 1.0 * float(p["dz"])))
    q.a_background = 1 if a_background else 0
    # non-uniform vertical grid: p["z"], the nz + 6 layer positions (k = -3 ..
    # nz + 2); the array stays referenced by the struct while it is in use
    if p.get("z") is not None:
        zarr = np.ascontiguousarray(p["z"], dtype=np.float64)
        if zarr.shape != (q.nz + 2 * NGHOST,):
            raise ValueError("p['z'] must hold nz + 6 layer positions")
        q.z = zarr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        q._zkeep = zarr
    return q


def fma_peak(precision: int, device: str = "cuda:0") -> float:
    """FMA throughput of the device in FP32 or FP64 (flop/s), measured by
    the library's probe kernel (mhd_fma_peak)."""
    import torch
    lib = load()
    scratch = torch.empty(1 << 16, dtype=torch.float64, device=device)
    out = ctypes.c_double()
    rc = lib.mhd_fma_peak(int(precision), ctypes.c_void_p(scratch.data_ptr()),
                          ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream), ctypes.byref(out))
    if rc != MHD_OK:
        raise MHDError(rc, lib.mhd_last_error(None).decode())
    return out.value


def _path(p) -> Optional[bytes]:
    return None if p is None else os.fsencode(p)


def h5_write(var_path, grid_path, params: Dict, t: float, padded=None, precision: int = 64):
    """Snapshot files in the paper's HDF5 layout from host data
    (mhd_h5_write): padded is the [8][nz+6][ny+6][nx+6] state in the given
    precision (numpy), or None when only grid_path is written."""
    lib = load()
    q = make_params(params, precision)
    keep = None
    ptr = None
    if padded is not None:
        keep = np.ascontiguousarray(padded, dtype=np.float64 if precision == 64 else np.float32)
        ng = NGHOST
        if keep.shape != (NFIELD, q.nz + 2 * ng, q.ny + 2 * ng, q.nx + 2 * ng):
            raise ValueError("padded must be [8][nz+6][ny+6][nx+6]")
        ptr = ctypes.c_void_p(keep.ctypes.data)
    rc = lib.mhd_h5_write(_path(var_path), _path(grid_path), ctypes.byref(q), float(t), ptr)
    if rc != MHD_OK:
        raise MHDError(rc, lib.mhd_last_error(None).decode())


def h5_checksum(data: bytes) -> int:
    """The lookup3 checksum the snapshot files carry (mhd_h5_checksum)."""
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    return int(load().mhd_h5_checksum(buf, len(data)))


def workspace_bytes(p: Dict, precision: int = 32, a_background: bool = False) -> int:
    q = make_params(p, precision, a_background=a_background)
    return int(load().mhd_workspace_bytes(ctypes.byref(q)))


class Simulation:
    """One libmhd handle.  Arrays passed in may be torch CUDA tensors
    (device pointers) or numpy arrays (host pointers); the element type must
    match the precision (float32 / float64).

    a_background: an FP64 [3][nz][ny][nx] field (numpy array or float64 CUDA
    tensor), typically the initial potential field.  A is then stored as a
    perturbation about it (mhd_set_a_background): the state's A fields are
    replaced by this background, with zero perturbation."""

    def __init__(self, params: Dict, init_state, lnrho0, lnT0=None, precision: int = 32,
                 stats_every: int = 0, device: str = "cuda:0", stream=None, adjoint: bool = False,
                 a_background=None):
        import torch
        self.lib = load()
        self.params = dict(params)
        self.precision = int(precision)
        self.np_dtype = np.float32 if precision == 32 else np.float64
        self.torch_dtype = torch.float32 if precision == 32 else torch.float64
        self.device = torch.device(device)
        self._p = make_params(params, precision, stats_every, adjoint, a_background is not None)
        nbytes = int(self.lib.mhd_workspace_bytes(ctypes.byref(self._p)))
        if nbytes == 0:
            raise MHDError(MHD_ERR_ARG, "invalid parameters")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._ws_bytes = nbytes
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        lr = np.ascontiguousarray(lnrho0, dtype=np.float64)
        if lr.shape != (self._p.nz + 2 * NGHOST,):
            raise ValueError("lnrho0 must have nz + 6 entries")
        lt = None
        if lnT0 is not None:
            lt = np.ascontiguousarray(lnT0, dtype=np.float64)
            if lt.shape != (self._p.nz + 2 * NGHOST,):
                raise ValueError("lnT0 must have nz + 6 entries")
        ptr, mem, keep = self._in(init_state, (NFIELD, self._p.nz, self._p.ny, self._p.nx))
        h = ctypes.c_void_p()
        rc = self.lib.mhd_create(ctypes.byref(self._p), ctypes.c_void_p(self._ws_ptr),
                                 ctypes.c_size_t(nbytes), ptr, mem,
                                 lr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 None if lt is None else lt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        del keep
        if rc != MHD_OK:
            raise MHDError(rc, self.lib.mhd_last_error(None).decode())
        self.h = h
        if a_background is not None:
            self.set_a_background(a_background)

    # -- marshalling --
    def _in(self, a, shape):
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_cuda:
                a = a.numpy()
            else:
                if a.dtype != self.torch_dtype or tuple(a.shape) != tuple(shape) or not a.is_contiguous():
                    raise ValueError(f"expected contiguous {self.torch_dtype} tensor of shape {shape}")
                return ctypes.c_void_p(a.data_ptr()), MHD_MEM_DEVICE, a
        arr = np.ascontiguousarray(a, dtype=self.np_dtype)
        if arr.shape != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {arr.shape}")
        return ctypes.c_void_p(arr.ctypes.data), MHD_MEM_HOST, arr

    def _check(self, rc):
        if rc != MHD_OK:
            raise MHDError(rc, self.lib.mhd_last_error(self.h).decode())

    # -- API --
    def set_a_background(self, a_bg, a_pert=None):
        """A = a_bg (FP64, [3][nz][ny][nx]) + a_pert (the handle's precision,
        or None for zero), stored as background and perturbation."""
        import torch
        shape = (3, self._p.nz, self._p.ny, self._p.nx)
        on_dev = lambda a: isinstance(a, torch.Tensor) and a.is_cuda
        # one mem flag for both arrays: a host array beside a device one is
        # copied to the device first
        if on_dev(a_pert) and not on_dev(a_bg):
            a_bg = torch.as_tensor(np.ascontiguousarray(a_bg, dtype=np.float64), device=self.device)
        elif on_dev(a_bg) and a_pert is not None and not on_dev(a_pert):
            a_pert = torch.as_tensor(np.ascontiguousarray(a_pert, dtype=self.np_dtype), device=self.device)
        if on_dev(a_bg):
            if a_bg.dtype != torch.float64 or tuple(a_bg.shape) != shape or not a_bg.is_contiguous():
                raise ValueError(f"a_bg must be a contiguous float64 tensor of shape {shape}")
            bp, mem, keep_b = ctypes.c_void_p(a_bg.data_ptr()), MHD_MEM_DEVICE, a_bg
        else:
            if isinstance(a_bg, torch.Tensor):
                a_bg = a_bg.numpy()
            keep_b = np.ascontiguousarray(a_bg, dtype=np.float64)
            if keep_b.shape != shape:
                raise ValueError(f"a_bg must have shape {shape}")
            bp, mem = ctypes.c_void_p(keep_b.ctypes.data), MHD_MEM_HOST
        pp, keep_p = None, None
        if a_pert is not None:
            pp, mp, keep_p = self._in(a_pert, shape)
            if mp != mem:
                raise ValueError("a_bg and a_pert must both be host arrays or both device tensors")
        self._check(self.lib.mhd_set_a_background(self.h, bp, pp, mem))
        del keep_b, keep_p

    def set_driver(self, bz, v0, v1, t0: float, t1: float):
        n = (self._p.ny, self._p.nx)
        b, mb, k1 = self._in(bz, n)
        a0, m0, k2 = self._in(v0, (2,) + n)
        a1, m1, k3 = self._in(v1, (2,) + n)
        if not (mb == m0 == m1):
            raise ValueError("bz, v0, v1 must all be host arrays or all device tensors")
        self._check(self.lib.mhd_set_driver(self.h, b, a0, a1, float(t0), float(t1), mb))

    def step(self, nsteps: int = 1):
        self._check(self.lib.mhd_step(self.h, int(nsteps)))

    def read(self, field: int = -1, out=None):
        import torch
        shape = ((NFIELD,) if field < 0 else ()) + (self._p.nz, self._p.ny, self._p.nx)
        if out is None:
            out = torch.empty(shape, dtype=self.torch_dtype, device=self.device)
        if isinstance(out, np.ndarray):
            self._check(self.lib.mhd_read(self.h, int(field), ctypes.c_void_p(out.ctypes.data), MHD_MEM_HOST))
        else:
            self._check(self.lib.mhd_read(self.h, int(field), ctypes.c_void_p(out.data_ptr()), MHD_MEM_DEVICE))
        return out

    def write_snapshot(self, var_path=None, grid_path=None):
        """var.h5 and/or grid.h5 of the current state in the paper's HDF5
        layout (mhd_write_snapshot; fills the ghosts first)."""
        self._check(self.lib.mhd_write_snapshot(self.h, _path(var_path), _path(grid_path)))

    def read_plane(self, field: int, k: int, out=None):
        """Layer k of one field, [ny][nx]; out: a numpy array (host) or a
        CUDA tensor (device), allocated on the device when None."""
        import torch
        if out is None:
            out = torch.empty((self._p.ny, self._p.nx), dtype=self.torch_dtype, device=self.device)
        if isinstance(out, np.ndarray):
            self._check(self.lib.mhd_read_plane(self.h, int(field), int(k), ctypes.c_void_p(out.ctypes.data),
                                                MHD_MEM_HOST))
        else:
            self._check(self.lib.mhd_read_plane(self.h, int(field), int(k), ctypes.c_void_p(out.data_ptr()),
                                                MHD_MEM_DEVICE))
        return out

    def write(self, state):
        ptr, mem, keep = self._in(state, (NFIELD, self._p.nz, self._p.ny, self._p.nx))
        self._check(self.lib.mhd_write(self.h, ptr, mem))

    def padded_shape(self):
        return (NFIELD, self._p.nz + 2 * NGHOST, self._p.ny + 2 * NGHOST, self._p.nx + 2 * NGHOST)

    def read_padded(self, which: int = 0) -> np.ndarray:
        out = np.empty(self.padded_shape(), dtype=self.np_dtype)
        self._check(self.lib.mhd_read_padded(self.h, int(which), ctypes.c_void_p(out.ctypes.data), MHD_MEM_HOST))
        return out

    def fill_ghosts(self):
        self._check(self.lib.mhd_fill_ghosts(self.h))

    def eval_rhs(self, t: float) -> np.ndarray:
        out = np.empty(self.padded_shape(), dtype=self.np_dtype)
        self._check(self.lib.mhd_eval_rhs(self.h, float(t), ctypes.c_void_p(out.ctypes.data), MHD_MEM_HOST))
        return out

    def compute_dt(self) -> float:
        dt = ctypes.c_double()
        self._check(self.lib.mhd_compute_dt(self.h, ctypes.byref(dt)))
        return dt.value

    def compute_stats(self) -> Dict:
        s = Stats()
        self._check(self.lib.mhd_compute_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def read_stats(self) -> Dict:
        s = Stats()
        self._check(self.lib.mhd_read_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def time(self):
        t, dt = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.mhd_get_time(self.h, ctypes.byref(t), ctypes.byref(dt)))
        return t.value, dt.value

    def read_target(self) -> np.ndarray:
        out = np.empty((2, self._p.ny, self._p.nx), dtype=self.np_dtype)
        self._check(self.lib.mhd_read_target(self.h, ctypes.c_void_p(out.ctypes.data), MHD_MEM_HOST))
        return out

    # -- adjoint --
    def set_time(self, t: float):
        self._check(self.lib.mhd_set_time(self.h, float(t)))

    def checkpoint_bytes(self) -> int:
        return int(self.lib.mhd_checkpoint_bytes(self.h))

    def new_checkpoint(self):
        import torch
        return torch.empty(self.checkpoint_bytes(), dtype=torch.uint8, device=self.device)

    def save(self, buf) -> float:
        t = ctypes.c_double()
        self._check(self.lib.mhd_save(self.h, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(t)))
        return t.value

    def restore(self, buf, t: float):
        self._check(self.lib.mhd_restore(self.h, ctypes.c_void_p(buf.data_ptr()), float(t)))

    def tape_bytes(self) -> int:
        return int(self.lib.mhd_tape_bytes(self.h))

    def new_tape(self):
        import torch
        return torch.empty(self.tape_bytes(), dtype=torch.uint8, device=self.device)

    def step_taped(self, tape):
        """One step that keeps its substep states (and start time) in `tape`."""
        self._check(self.lib.mhd_step_taped(self.h, ctypes.c_void_p(tape.data_ptr())))

    def adjoint_step_taped(self, tape):
        """The reverse step of the step recorded in `tape`."""
        self._check(self.lib.mhd_adjoint_step_taped(self.h, ctypes.c_void_p(tape.data_ptr())))

    def adjoint_init(self, lam):
        ptr, mem, keep = self._in(lam, (NFIELD, self._p.nz, self._p.ny, self._p.nx))
        self._check(self.lib.mhd_adjoint_init(self.h, ptr, mem))

    def adjoint_step(self):
        self._check(self.lib.mhd_adjoint_step(self.h))

    def adjoint_read(self) -> Dict:
        import torch
        n = (self._p.ny, self._p.nx)
        out = {"lam": torch.empty((NFIELD, self._p.nz) + n, dtype=self.torch_dtype, device=self.device),
               "bz": torch.empty(n, dtype=self.torch_dtype, device=self.device),
               "v0": torch.empty((2,) + n, dtype=self.torch_dtype, device=self.device),
               "v1": torch.empty((2,) + n, dtype=self.torch_dtype, device=self.device)}
        self._check(self.lib.mhd_adjoint_read(self.h, *(ctypes.c_void_p(out[k].data_ptr()) for k in
                                                        ("lam", "bz", "v0", "v1")), MHD_MEM_DEVICE))
        return out

    def bz_plane(self, state, k: int):
        import torch
        st = state.contiguous()
        out = torch.empty((self._p.ny, self._p.nx), dtype=self.torch_dtype, device=self.device)
        self._check(self.lib.mhd_bz_plane(self.h, ctypes.c_void_p(st.data_ptr()), int(k),
                                          ctypes.c_void_p(out.data_ptr())))
        return out

    def bz_plane_adjoint(self, bbar, k: int):
        import torch
        bb = bbar.contiguous()
        lam = torch.empty((NFIELD, self._p.nz, self._p.ny, self._p.nx), dtype=self.torch_dtype, device=self.device)
        self._check(self.lib.mhd_bz_plane_adjoint(self.h, ctypes.c_void_p(bb.data_ptr()), int(k),
                                                  ctypes.c_void_p(lam.data_ptr())))
        return lam

    def profile(self, enable=True):
        """True / 1: record class times as the step runs; 2: record with every
        kernel serialised on the handle's stream; False / 0: stop."""
        mode = 0 if enable is False else (1 if enable is True else int(enable))
        self._check(self.lib.mhd_profile(self.h, mode))

    def read_profile(self) -> Dict:
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        n = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        self._check(self.lib.mhd_read_profile(self.h, ms, n))
        return {c: (ms[q], n[q]) for q, c in enumerate(KERNEL_CLASSES)}

    def debug_skip_copy(self, plane: int, wait_limit: int):
        """Test hook of the bounded waits (mhd_debug_skip_copy)."""
        self._check(self.lib.mhd_debug_skip_copy(self.h, int(plane), int(wait_limit)))

    def launch_count(self) -> int:
        return int(self.lib.mhd_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
