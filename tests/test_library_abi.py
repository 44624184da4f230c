"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/mhd.h declares; argument errors come back before any
launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_08557_gb300 import build as _b  # noqa: F401
    from paper_1908_08557_gb300.build import build
    from paper_1908_08557_gb300 import binding
    build()
    return binding.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhd_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_sizing_and_argument_errors(lib):
    import inputs
    from paper_1908_08557_gb300 import binding
    p = inputs.scheme_params(32, 32, 32)
    q = binding.make_params(p, 32)
    n32 = lib.mhd_workspace_bytes(ctypes.byref(q))
    q64 = binding.make_params(p, 64)
    n64 = lib.mhd_workspace_bytes(ctypes.byref(q64))
    # three padded state sets dominate: 8 fields x 38 x 38 x 40 cells
    assert n32 > 3 * 8 * 38 * 38 * 40 * 4 and n64 > n32
    bad = binding.make_params(dict(p, nx=48), 32)      # not a power of two with the FFT boundary
    assert lib.mhd_workspace_bytes(ctypes.byref(bad)) == 0
    ok_periodic = binding.make_params(dict(p, nx=48, bc_z=1), 32)
    assert lib.mhd_workspace_bytes(ctypes.byref(ok_periodic)) > 0
    bad = binding.make_params(dict(p), 16)             # precision
    assert lib.mhd_workspace_bytes(ctypes.byref(bad)) == 0
    h = ctypes.c_void_p()
    lr = (ctypes.c_double * 38)()
    rc = lib.mhd_create(ctypes.byref(q), None, 0, ctypes.c_void_p(1), 0, lr, None, None, ctypes.byref(h))
    assert rc == binding.MHD_ERR_WORKSPACE and not h.value
    assert b"workspace" in lib.mhd_last_error(None)
    rc = lib.mhd_create(ctypes.byref(bad), ctypes.c_void_p(256), 1 << 30, ctypes.c_void_p(1), 0, lr, None,
                        None, ctypes.byref(h))
    assert rc == binding.MHD_ERR_ARG
    rc = lib.mhd_create(ctypes.byref(q), ctypes.c_void_p(256 + 8), 1 << 40, ctypes.c_void_p(1), 0, lr, None,
                        None, ctypes.byref(h))
    assert rc == binding.MHD_ERR_WORKSPACE   # misaligned
    assert lib.mhd_step(None, 1) == binding.MHD_ERR_ARG


def test_background_and_vertical_grid_parameters(lib):
    """Workspace sizing with A stored about a background (more tables) and
    with a non-uniform vertical grid; neither combines with the adjoint; the
    positions must increase strictly."""
    import numpy as np

    import inputs
    from paper_1908_08557_gb300 import binding
    p = inputs.scheme_params(32, 32, 24)
    n = lib.mhd_workspace_bytes(ctypes.byref(binding.make_params(p, 32)))
    nb = lib.mhd_workspace_bytes(ctypes.byref(binding.make_params(p, 32, a_background=True)))
    assert nb > n > 0
    bad = binding.make_params(p, 32, adjoint=True, a_background=True)
    assert lib.mhd_workspace_bytes(ctypes.byref(bad)) == 0
    z, _, _ = inputs.stretched_z(24, 0.5, 1.5, 12, 4)
    qz = binding.make_params(dict(p, z=z), 32)
    assert lib.mhd_workspace_bytes(ctypes.byref(qz)) > 0
    assert lib.mhd_workspace_bytes(ctypes.byref(binding.make_params(dict(p, z=z), 32, adjoint=True))) == 0
    zbad = z.copy()
    zbad[10] = zbad[9]
    assert lib.mhd_workspace_bytes(ctypes.byref(binding.make_params(dict(p, z=zbad), 32))) == 0
    assert lib.mhd_workspace_bytes(ctypes.byref(binding.make_params(dict(p, z=z[::-1].copy()), 64))) == 0
    with np.testing.assert_raises(ValueError):
        binding.make_params(dict(p, z=z[:-1]), 32)


def test_cooling_parameter_errors(lib):
    """Newtonian cooling (Sect. 3.1): invalid rates and cut-off widths are
    rejected before any allocation, and so is an initial ln rho profile that
    does not fall strictly with height (its inverse is the lookup of T')."""
    import inputs
    from paper_1908_08557_gb300 import binding
    p = inputs.scheme_params(32, 32, 32, nc_tau=0.5)
    ok = binding.make_params(p, 32)
    assert lib.mhd_workspace_bytes(ctypes.byref(ok)) > 0
    for over in (dict(nc_tau=-0.1), dict(nc_lnrho_width=9.0), dict(nc_lnrho_width=0.0), dict(nc_z_width=0.0)):
        bad = binding.make_params(dict(p, **over), 32)
        assert lib.mhd_workspace_bytes(ctypes.byref(bad)) == 0, over
    h = ctypes.c_void_p()
    flat = (ctypes.c_double * 38)()  # ln rho0 = 0 everywhere: not strictly falling
    rc = lib.mhd_create(ctypes.byref(ok), ctypes.c_void_p(256), 1 << 40, ctypes.c_void_p(1), 0, flat, None, None,
                        ctypes.byref(h))
    assert rc == binding.MHD_ERR_ARG and not h.value
    assert b"falling strictly" in lib.mhd_last_error(None)


def test_granulation_argument_errors(lib):
    """The granulation driver (Sect. 2.3): workspace sizing, and every
    argument error returned before any CUDA call."""
    from paper_1908_08557_gb300 import binding
    from paper_1908_08557_gb300.granulation import paper_params
    gp = binding.GranParams(**paper_params(mm_per_unit=0.23))
    n256 = lib.mhd_gran_workspace_bytes(256, 256, 1.0, 1.0, ctypes.byref(gp))
    n1k = lib.mhd_gran_workspace_bytes(1024, 1024, 1.0, 1.0, ctypes.byref(gp))
    # 132 bytes per pixel (granule slots, placement state, fields, staged
    # draws, two complex FFT planes) plus small tables
    assert 132 * 256 * 256 <= n256 < 132 * 256 * 256 + (1 << 20)
    assert 132 * 1024 * 1024 <= n1k < 132 * 1024 * 1024 + (1 << 20)
    bad = [(48, 256, 1.0, 1.0, {}),                      # not a power of two
           (2048, 256, 1.0, 1.0, {}),                    # beyond the FFT's 1024
           (8, 8, 1.0, 1.0, {}),                         # lane radius above half the plane
           (256, 256, 0.0, 1.0, {}),                     # spacing
           (256, 256, 0.01, 1.0, {}),                    # lane radius beyond 64 pixels
           (256, 256, 1.0, 1.0, dict(r_lane=3.0)),       # r_lane below r_granule
           (256, 256, 1.0, 1.0, dict(vmin_frac=0.9)),    # v_min above the lowest v_max
           (256, 256, 1.0, 1.0, dict(amp_spread=1.0)),
           (256, 256, 1.0, 1.0, dict(lifetime=0.0)),
           (256, 256, 1.0, 1.0, dict(f_rot=float("nan")))]
    for nx, ny, dx, dy, over in bad:
        q = binding.GranParams(**dict(paper_params(mm_per_unit=0.23), **over))
        assert lib.mhd_gran_workspace_bytes(nx, ny, dx, dy, ctypes.byref(q)) == 0, (nx, ny, dx, over)
    h = ctypes.c_void_p()
    rc = lib.mhd_gran_create(256, 256, 1.0, 1.0, ctypes.byref(gp), None, 0, None, ctypes.byref(h))
    assert rc == binding.MHD_ERR_WORKSPACE and not h.value
    assert b"workspace" in lib.mhd_gran_last_error(None)
    rc = lib.mhd_gran_create(256, 256, 1.0, 1.0, ctypes.byref(gp), ctypes.c_void_p(256 + 8), 1 << 40, None,
                             ctypes.byref(h))
    assert rc == binding.MHD_ERR_WORKSPACE
    rc = lib.mhd_gran_create(48, 256, 1.0, 1.0, ctypes.byref(gp), ctypes.c_void_p(256), 1 << 40, None,
                             ctypes.byref(h))
    assert rc == binding.MHD_ERR_ARG and b"powers of two" in lib.mhd_gran_last_error(None)
    assert lib.mhd_gran_create(256, 256, 1.0, 1.0, ctypes.byref(gp), ctypes.c_void_p(256), 1 << 40, None,
                               None) == binding.MHD_ERR_ARG
    r = ctypes.c_int()
    assert lib.mhd_gran_update(None, 0.0, None, None, None, 0, ctypes.byref(r)) == binding.MHD_ERR_ARG
    assert lib.mhd_gran_velocity(None, 0.0, 32, None, 0) == binding.MHD_ERR_ARG
    assert lib.mhd_gran_read_granules(None, None, None, 0) == binding.MHD_ERR_ARG
    assert lib.mhd_gran_read_field(None, 0, None, 0) == binding.MHD_ERR_ARG
    assert lib.mhd_gran_launch_count(None) == 0
    lib.mhd_gran_destroy(None)


def test_null_handle_is_an_argument_error(lib):
    """Every entry point that takes a handle (or a granulation generator)
    answers a NULL one with MHD_ERR_ARG before touching the device: size and
    count queries with 0, the error-message queries with a message, the
    destroy calls with nothing.  Argument types follow the header."""
    from paper_1908_08557_gb300 import binding
    own = ctypes.CDLL(lib._name)  # own function objects: the binding's argtypes stay as they are
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    decls = re.findall(r"([A-Za-z_][\w\s\*]*?)\b(mhd_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S)

    def arg(a):
        a = a.strip()
        if "*" in a or a.startswith(("mhd_handle", "mhd_gran_handle")):
            return ctypes.c_void_p, None
        if a.startswith("double"):
            return ctypes.c_double, 0.0
        if a.startswith("size_t"):
            return ctypes.c_size_t, 0
        if a.startswith("long long"):
            return ctypes.c_longlong, 0
        return ctypes.c_int, 0

    seen = 0
    for ret, name, args in decls:
        params = [x for x in " ".join(args.split()).split(",") if x.strip()]
        if not params or not params[0].strip().startswith(("mhd_handle", "mhd_gran_handle")):
            continue
        f = getattr(own, name)
        spec = [arg(p) for p in params]
        f.argtypes = [t for t, _ in spec]
        r = " ".join(ret.split())
        kind = "msg" if "char" in r else "size" if r in ("size_t", "long long") else "void" if r == "void" else "rc"
        f.restype = {"msg": ctypes.c_char_p, "size": ctypes.c_longlong, "void": None, "rc": ctypes.c_int}[kind]
        out = f(*[v for _, v in spec])
        if kind == "rc":
            assert out == binding.MHD_ERR_ARG, (name, out)
        elif kind == "size":
            assert out == 0, (name, out)
        elif kind == "msg":
            assert out, name
        seen += 1
    assert seen >= 35
