"""A small reader of HDF5 files, written for the tests from the HDF5 file
format specification (version 3): superblock versions 2 and 3, version 2
object headers (single chunk), groups stored compactly as Link messages,
datasets with contiguous or compact layout and fixed-point, IEEE
floating-point or fixed-length string datatypes.  Every superblock and
object-header checksum is verified.

It shares nothing with the library's writer; no HDF5 library is installed
where the tests run, so this reader is what the snapshot files are checked
against.  Anything outside that subset raises ValueError.
"""
import struct

import numpy as np

SIGNATURE = b"\x89HDF\r\n\x1a\n"
UNDEF = 0xFFFFFFFFFFFFFFFF


def lookup3(data: bytes, initval: int = 0) -> int:
    """Bob Jenkins' lookup3 hashlittle (byte-wise form), 32-bit result."""
    M = 0xFFFFFFFF

    def rot(x, k):
        return ((x << k) | (x >> (32 - k))) & M

    n = len(data)
    a = b = c = (0xDEADBEEF + n + initval) & M
    i = 0
    while n - i > 12:
        a = (a + int.from_bytes(data[i:i + 4], "little")) & M
        b = (b + int.from_bytes(data[i + 4:i + 8], "little")) & M
        c = (c + int.from_bytes(data[i + 8:i + 12], "little")) & M
        a = (a - c) & M; a ^= rot(c, 4); c = (c + b) & M
        b = (b - a) & M; b ^= rot(a, 6); a = (a + c) & M
        c = (c - b) & M; c ^= rot(b, 8); b = (b + a) & M
        a = (a - c) & M; a ^= rot(c, 16); c = (c + b) & M
        b = (b - a) & M; b ^= rot(a, 19); a = (a + c) & M
        c = (c - b) & M; c ^= rot(b, 4); b = (b + a) & M
        i += 12
    rest = data[i:]
    if not rest:
        return c
    rest = rest + bytes(12 - len(rest))
    a = (a + int.from_bytes(rest[0:4], "little")) & M
    b = (b + int.from_bytes(rest[4:8], "little")) & M
    c = (c + int.from_bytes(rest[8:12], "little")) & M
    c ^= b; c = (c - rot(b, 14)) & M
    a ^= c; a = (a - rot(c, 11)) & M
    b ^= a; b = (b - rot(a, 25)) & M
    c ^= b; c = (c - rot(b, 16)) & M
    a ^= c; a = (a - rot(c, 4)) & M
    b ^= a; b = (b - rot(a, 14)) & M
    c ^= b; c = (c - rot(b, 24)) & M
    return c


class File:
    """Parsed file: `root` is a dict name -> dict (group) or numpy array /
    bytes (dataset); `objects` counts the object headers read."""

    def __init__(self, path):
        with open(path, "rb") as f:
            self.buf = f.read()
        self.objects = 0
        self._superblock()
        self.root = self._object(self.root_addr)

    # -- helpers --------------------------------------------------------
    def _u(self, at, n):
        return int.from_bytes(self.buf[at:at + n], "little")

    def _superblock(self):
        b = self.buf
        if b[:8] != SIGNATURE:
            raise ValueError("not an HDF5 file (signature)")
        version = b[8]
        if version not in (2, 3):
            raise ValueError(f"superblock version {version} not supported")
        self.so, self.sl = b[9], b[10]
        if (self.so, self.sl) != (8, 8):
            raise ValueError("only 8-byte offsets and lengths")
        p = 12
        base, ext, eof, root = (self._u(p + 8 * q, 8) for q in range(4))
        p += 32
        if lookup3(b[:p]) != self._u(p, 4):
            raise ValueError("superblock checksum")
        if base != 0:
            raise ValueError("base address must be 0")
        if ext != UNDEF:
            raise ValueError("superblock extension not supported")
        if eof != len(b):
            raise ValueError(f"end-of-file address {eof} != file size {len(b)}")
        self.superblock_size = p + 4
        self.root_addr = root

    def _messages(self, at):
        b = self.buf
        if b[at:at + 4] != b"OHDR":
            raise ValueError(f"object header signature at {at}")
        if b[at + 4] != 2:
            raise ValueError("object header version")
        flags = b[at + 5]
        p = at + 6
        if flags & 0x20:
            p += 16                  # access, modification, change, birth times
        if flags & 0x10:
            p += 4                   # attribute phase change values
        w = 1 << (flags & 3)
        chunk = self._u(p, w)
        p += w
        end = p + chunk
        if lookup3(b[at:end]) != self._u(end, 4):
            raise ValueError(f"object header checksum at {at}")
        self.objects += 1
        msgs = []
        while end - p >= 4:
            mtype, size, mflags = b[p], self._u(p + 1, 2), b[p + 3]
            p += 4
            if flags & 0x04:
                p += 2               # creation order
            msgs.append((mtype, b[p:p + size]))
            p += size
        return msgs

    def _object(self, at):
        msgs = self._messages(at)
        types = [t for t, _ in msgs]
        if 0x0002 in types or 0x0006 in types:
            if 0x0002 not in types:
                raise ValueError("group without a Link Info message")
            out = {}
            for t, m in msgs:
                if t == 0x0002:
                    if m[0] != 0:
                        raise ValueError("link info version")
                    q = 2 + (8 if m[1] & 1 else 0)
                    heap = int.from_bytes(m[q:q + 8], "little")
                    if heap != UNDEF:
                        raise ValueError("dense link storage not supported")
                elif t == 0x0006:
                    name, addr = self._link(m)
                    out[name] = self._object(addr)
            return out
        return self._dataset(msgs)

    @staticmethod
    def _link(m):
        if m[0] != 1:
            raise ValueError("link message version")
        fl = m[1]
        p = 2
        ltype = 0
        if fl & 0x08:
            ltype = m[p]
            p += 1
        if fl & 0x04:
            p += 8
        if fl & 0x10:
            if m[p] != 0:
                raise ValueError("only ASCII link names")
            p += 1
        w = 1 << (fl & 3)
        n = int.from_bytes(m[p:p + w], "little")
        p += w
        name = m[p:p + n].decode("ascii")
        p += n
        if ltype != 0:
            raise ValueError("only hard links")
        return name, int.from_bytes(m[p:p + 8], "little")

    def _dataset(self, msgs):
        shape = dtype = data = None
        for t, m in msgs:
            if t == 0x0001:
                ver, nd, fl = m[0], m[1], m[2]
                if ver == 2:
                    dstype = m[3]
                    p = 4
                elif ver == 1:
                    dstype = 1 if nd else 0
                    p = 8
                else:
                    raise ValueError("dataspace version")
                if dstype == 2:
                    raise ValueError("null dataspace")
                shape = tuple(int.from_bytes(m[p + 8 * q:p + 8 * q + 8], "little") for q in range(nd))
            elif t == 0x0003:
                dtype = self._dtype(m)
            elif t == 0x0008:
                if m[0] != 3:
                    raise ValueError("layout version")
                if m[1] == 1:
                    addr = int.from_bytes(m[2:10], "little")
                    size = int.from_bytes(m[10:18], "little")
                    data = self.buf[addr:addr + size]
                    if len(data) != size:
                        raise ValueError("raw data beyond the end of the file")
                elif m[1] == 0:
                    size = int.from_bytes(m[2:4], "little")
                    data = m[4:4 + size]
                else:
                    raise ValueError("chunked layout not supported")
        if shape is None or dtype is None or data is None:
            raise ValueError("dataset without dataspace, datatype or layout")
        if dtype == "string":
            return bytes(data)
        n = int(np.prod(shape)) if shape else 1
        if len(data) != n * dtype.itemsize:
            raise ValueError("raw data size does not match dataspace x datatype")
        arr = np.frombuffer(data, dtype=dtype).reshape(shape)
        return arr

    @staticmethod
    def _dtype(m):
        cls, ver = m[0] & 0x0F, m[0] >> 4
        if ver != 1:
            raise ValueError("datatype version")
        bits = m[1] | (m[2] << 8) | (m[3] << 16)
        size = int.from_bytes(m[4:8], "little")
        if cls == 1:
            if bits & 1:
                raise ValueError("big-endian float")
            offset, prec = struct.unpack_from("<HH", m, 8)
            eloc, esize, mloc, msize = m[12], m[13], m[14], m[15]
            bias = int.from_bytes(m[16:20], "little")
            ieee = {4: (32, 23, 8, 0, 23, 127, 31), 8: (64, 52, 11, 0, 52, 1023, 63)}
            want = ieee.get(size)
            if want is None or (prec, eloc, esize, mloc, msize, bias, (bits >> 8) & 0xFF) != want or offset != 0:
                raise ValueError("not an IEEE float layout")
            if (bits >> 4) & 3 != 2:
                raise ValueError("mantissa normalisation")
            return np.dtype("<f4" if size == 4 else "<f8")
        if cls == 0:
            if bits & 1:
                raise ValueError("big-endian integer")
            signed = bool(bits & 0x08)
            offset, prec = struct.unpack_from("<HH", m, 8)
            if offset != 0 or prec != 8 * size:
                raise ValueError("integer bit layout")
            return np.dtype(("<i" if signed else "<u") + str(size))
        if cls == 3:
            return "string"
        raise ValueError(f"datatype class {cls} not supported")
