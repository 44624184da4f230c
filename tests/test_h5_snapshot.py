"""Snapshot files in the layout of the paper's HDF5 snapshots (Sect. 5.3:
var.h5 with the groups data / grid / settings and the scalar time, grid.h5
with the global grid, settings/precision "S" or "D", arrays read as Fortran
(x, y, z) with the outer ghost layers kept), written by the library from
host data (mhd_h5_write; no CUDA call) and read back by tests/h5read.py, a
reader written separately from the HDF5 file format specification.

The checksum both sides use is pinned to the published lookup3 test values;
the grid to closed forms.  No HDF5 library is installed here or on the GPU
machine: the h5py cross-check runs only where h5py is importable.
"""
import os

import numpy as np
import pytest

import h5read
import inputs

NG = 3
NAMES = ["ax", "ay", "az", "ux", "uy", "uz", "lnrho", "lnTT"]


@pytest.fixture(scope="module")
def binding():
    from paper_1908_08557_gb300 import binding as b
    from paper_1908_08557_gb300.build import build
    build()
    b.load()
    return b


def test_lookup3_published_values(binding):
    """Bob Jenkins' published results of hashlittle: the empty key gives
    the initial state 0xdeadbeef + initval; "Four score and seven years ago"
    (30 bytes) gives 0x17770551 (initval 0) and 0xcd628161 (initval 1)."""
    key = b"Four score and seven years ago"
    assert h5read.lookup3(b"", 0) == 0xDEADBEEF
    assert h5read.lookup3(b"", 0xDEADBEEF) == 0xBD5B7DDE
    assert h5read.lookup3(key, 0) == 0x17770551
    assert h5read.lookup3(key, 1) == 0xCD628161
    assert binding.h5_checksum(b"") == 0xDEADBEEF
    assert binding.h5_checksum(key) == 0x17770551
    # the library's and the reader's versions agree on every tail length
    rng = np.random.default_rng(5)
    for n in list(range(0, 40)) + [97, 1000]:
        data = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert binding.h5_checksum(data) == h5read.lookup3(data), n


def _case(nx, ny, nz, seed, z=None):
    c = inputs.make_box(nx, ny, nz, seed=seed, z=z)
    return c.params


@pytest.mark.parametrize("precision", [64, 32])
def test_var_and_grid_files(binding, tmp_path, precision):
    p = _case(16, 8, 12, 3)
    rng = np.random.default_rng(7)
    dt = np.float64 if precision == 64 else np.float32
    padded = rng.standard_normal((8, 12 + 2 * NG, 8 + 2 * NG, 16 + 2 * NG)).astype(dt)
    var, grid = tmp_path / "var.h5", tmp_path / "grid.h5"
    binding.h5_write(var, grid, p, 1.25, padded, precision)

    raw = open(var, "rb").read()
    assert raw[:8] == b"\x89HDF\r\n\x1a\n" and raw[8] == 2
    f = h5read.File(var)
    assert f.superblock_size == 48
    assert set(f.root) == {"time", "data", "grid", "settings"}
    assert f.root["time"].shape == () and f.root["time"].dtype == np.float64 and f.root["time"] == 1.25
    assert list(f.root["data"]) == NAMES
    for q, name in enumerate(NAMES):
        a = f.root["data"][name]
        assert a.dtype == np.dtype(dt) and a.shape == (12 + 2 * NG, 8 + 2 * NG, 16 + 2 * NG)
        assert np.array_equal(a, padded[q])
        # Fortran view (x, y, z): the first index runs along x
        assert np.array_equal(a.T[:, 2, 5], padded[q, 5, 2, :])
    s = f.root["settings"]
    assert s["precision"] == (b"D" if precision == 64 else b"S")
    for k, v in (("nghost", NG), ("nx", 16), ("ny", 8), ("nz", 12), ("mx", 22), ("my", 14), ("mz", 18)):
        assert s[k].dtype == np.int32 and int(s[k]) == v, k
    g = f.root["grid"]
    i = np.arange(-NG, 16 + NG)
    assert np.array_equal(g["x"], i * p["dx"])
    assert np.array_equal(g["y"], np.arange(-NG, 8 + NG) * p["dy"])
    assert np.array_equal(g["z"], np.arange(-NG, 12 + NG) * p["dz"])
    assert np.array_equal(g["dx_1"], np.full(22, 1.0 / p["dx"]))
    assert np.allclose(g["dz_1"], 1.0 / p["dz"], rtol=1e-13, atol=0)
    assert float(g["dz"]) == pytest.approx(p["dz"], rel=1e-15)
    assert float(g["Lx"]) == 16 * p["dx"] and float(g["Ly"]) == 8 * p["dy"]
    assert float(g["Lz"]) == pytest.approx(12 * p["dz"], rel=1e-15)

    gf = h5read.File(grid)
    assert set(gf.root) == {"grid", "settings"}
    for k in g:
        assert np.array_equal(gf.root["grid"][k], g[k]), k
    # metadata precede the data; nothing but the nine datasets' bytes follows
    data_bytes = 8 * padded[0].nbytes
    assert len(raw) - data_bytes < 8192
    assert f.objects == 1 + 1 + 8 + 1 + 12 + 1 + 8 + 1  # root, time, data, 8 fields, grid + 12, settings + 8


def test_stretched_grid_inverse_spacing(binding, tmp_path):
    """dz_1 on a non-uniform grid: at interior layers the inverse of the
    sixth-order dz/dk of the positions (against the closed-form z'(k) of the
    generator), second order at the ghost layers."""
    z, zp, _ = inputs.stretched_z(24, 0.5, 1.5, 12, 4)
    p = _case(8, 8, 24, 4, z=z)
    binding.h5_write(None, tmp_path / "grid.h5", p, 0.0)
    g = h5read.File(tmp_path / "grid.h5").root["grid"]
    assert np.array_equal(g["z"], z)
    inner = slice(NG, 24 + NG)
    assert np.allclose(g["dz_1"][inner], 1.0 / zp[inner], rtol=1e-4, atol=0)
    assert np.allclose(g["dz_1"], 1.0 / zp, rtol=3e-2, atol=0)
    assert float(g["dz"]) == pytest.approx((z[24 + NG - 1] - z[NG]) / 23, rel=1e-14)


def test_errors(binding, tmp_path):
    p = _case(8, 8, 8, 5)
    with pytest.raises(binding.MHDError) as e:
        binding.h5_write(tmp_path / "no_such_dir" / "var.h5", None, p, 0.0, np.zeros((8, 14, 14, 14)))
    assert e.value.code == binding.MHD_ERR_IO
    with pytest.raises(binding.MHDError) as e:
        binding.h5_write(None, None, p, 0.0)
    assert e.value.code == binding.MHD_ERR_ARG
    with pytest.raises(ValueError):
        binding.h5_write(tmp_path / "v.h5", None, p, 0.0, np.zeros((8, 14, 14, 13)))


def test_reader_rejects_a_corrupted_file(binding, tmp_path):
    """A flipped byte in an object header or in the superblock fails its
    checksum (so the reader's checks are live)."""
    p = _case(8, 8, 8, 6)
    path = tmp_path / "g.h5"
    binding.h5_write(None, path, p, 0.0)
    raw = bytearray(open(path, "rb").read())
    for at in (20, 60):
        bad = bytearray(raw)
        bad[at] ^= 0x01
        bp = tmp_path / f"bad{at}.h5"
        open(bp, "wb").write(bytes(bad))
        with pytest.raises(ValueError):
            h5read.File(bp)


def test_h5py_reads_the_files(binding, tmp_path):
    h5py = pytest.importorskip("h5py")
    p = _case(8, 8, 8, 7)
    padded = np.random.default_rng(9).standard_normal((8, 14, 14, 14))
    binding.h5_write(tmp_path / "var.h5", None, p, 2.5, padded, 64)
    with h5py.File(tmp_path / "var.h5", "r") as f:
        assert float(f["time"][()]) == 2.5
        for q, name in enumerate(NAMES):
            assert np.array_equal(f["data"][name][()], padded[q])
        assert f["settings/precision"][()] == b"D"
