// mhd_h5.cu -- snapshot files in the layout of the paper's HDF5 snapshots
// (Sect. 5.3): `var.h5` with the time as a scalar FP64 dataset, the groups
// `data` (one dataset per variable, outer ghost layers kept, array order
// [z][y][x] with x fastest, i.e. Fortran (x, y, z)), `grid` and `settings`
// (with `precision` = "S" or "D"); `grid.h5` with the global grid (positions,
// spacings and their inverses, including `dz_1` of a non-uniform z grid).
//
// Host code only.  No HDF5 library is used: the files are written directly
// in the HDF5 file format (format specification version 3), in its
// simplest form that the library reads since version 1.8:
//   - superblock version 2 (48 bytes, no superblock extension),
//   - version 2 object headers ("OHDR"), one chunk each, no times,
//   - groups with compact link storage (Link Info, Group Info and one Link
//     message per member; no heaps, no B-trees),
//   - datasets with a version 2 dataspace, an IEEE little-endian float,
//     little-endian signed integer or fixed-length ASCII string datatype,
//     a version 3 fill value message and contiguous version 3 layout,
//   - every superblock and object header closed by the Jenkins lookup3
//     checksum (hashlittle, initial value 0) of its preceding bytes.
// Metadata come first, then the raw data of each dataset in the same order.
#include "../../include/mhd.h"
#include "mhd_internal.h"

#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

namespace mhd {
namespace h5w {

// ---- Jenkins lookup3 (hashlittle, byte-wise) -------------------------------
static inline uint32_t rot(uint32_t x, int k) { return (x << k) | (x >> (32 - k)); }

uint32_t lookup3(const void* key, size_t length, uint32_t initval) {
  const uint8_t* k = static_cast<const uint8_t*>(key);
  uint32_t a, b, c;
  a = b = c = 0xdeadbeefu + (uint32_t)length + initval;
  auto word = [](const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
  };
  while (length > 12) {
    a += word(k);
    b += word(k + 4);
    c += word(k + 8);
    // mix
    a -= c; a ^= rot(c, 4);  c += b;
    b -= a; b ^= rot(a, 6);  a += c;
    c -= b; c ^= rot(b, 8);  b += a;
    a -= c; a ^= rot(c, 16); c += b;
    b -= a; b ^= rot(a, 19); a += c;
    c -= b; c ^= rot(b, 4);  b += a;
    length -= 12;
    k += 12;
  }
  if (length == 0) return c;
  // the last 1..12 bytes, little-endian into a, b, c
  uint8_t tail[12] = {0};
  std::memcpy(tail, k, length);
  a += word(tail);
  b += word(tail + 4);
  c += word(tail + 8);
  // final
  c ^= b; c -= rot(b, 14);
  a ^= c; a -= rot(c, 11);
  b ^= a; b -= rot(a, 25);
  c ^= b; c -= rot(b, 16);
  a ^= c; a -= rot(c, 4);
  b ^= a; b -= rot(a, 14);
  c ^= b; c -= rot(b, 24);
  return c;
}

// ---- object tree -----------------------------------------------------------
enum TClass { T_INT = 0, T_FLOAT = 1, T_STRING = 3 };

struct Obj {
  bool group = true;
  std::string name;
  std::vector<Obj> kids;
  // dataset
  TClass tclass = T_FLOAT;
  int esize = 8;
  std::vector<uint64_t> dims;  // empty: scalar
  std::function<bool(FILE*)> emit;
  std::vector<uint8_t> small;  // raw bytes of a small dataset (emit unset)
  uint64_t ohdr = 0, data = 0;
  uint64_t nbytes() const {
    uint64_t n = (uint64_t)esize;
    for (uint64_t d : dims) n *= d;
    return n;
  }
};

static const uint64_t UNDEF = ~0ull;
// message types (format specification IV.A.2)
enum { M_DATASPACE = 0x0001, M_LINFO = 0x0002, M_DTYPE = 0x0003, M_FILL = 0x0005, M_LINK = 0x0006,
       M_LAYOUT = 0x0008, M_GINFO = 0x000A };

struct Buf {
  std::vector<uint8_t> v;
  void u8(unsigned x) { v.push_back((uint8_t)x); }
  void u16(unsigned x) { u8(x & 0xff); u8((x >> 8) & 0xff); }
  void u32(uint32_t x) { for (int i = 0; i < 4; ++i) u8((x >> (8 * i)) & 0xff); }
  void u64(uint64_t x) { for (int i = 0; i < 8; ++i) u8((unsigned)((x >> (8 * i)) & 0xff)); }
  void raw(const void* p, size_t n) { const uint8_t* q = (const uint8_t*)p; v.insert(v.end(), q, q + n); }
};

// message bodies of an object (addresses of the children must be set)
static std::vector<std::pair<int, Buf>> messages(const Obj& o) {
  std::vector<std::pair<int, Buf>> m;
  if (o.group) {
    Buf li;  // Link Info v0: no creation order; compact storage (no heap, no index)
    li.u8(0);
    li.u8(0);
    li.u64(UNDEF);
    li.u64(UNDEF);
    m.push_back({M_LINFO, li});
    Buf gi;  // Group Info v0, defaults
    gi.u8(0);
    gi.u8(0);
    m.push_back({M_GINFO, gi});
    for (const Obj& c : o.kids) {
      Buf lk;  // Link v1: hard link, one-byte name length, ASCII
      lk.u8(1);
      lk.u8(0);
      lk.u8((unsigned)c.name.size());
      lk.raw(c.name.data(), c.name.size());
      lk.u64(c.ohdr);
      m.push_back({M_LINK, lk});
    }
    return m;
  }
  Buf ds;  // Dataspace v2
  ds.u8(2);
  ds.u8((unsigned)o.dims.size());
  ds.u8(0);
  ds.u8(o.dims.empty() ? 0 : 1);
  for (uint64_t d : o.dims) ds.u64(d);
  m.push_back({M_DATASPACE, ds});
  Buf dt;  // Datatype v1
  if (o.tclass == T_FLOAT) {
    const bool dbl = o.esize == 8;
    dt.u8(0x10 | T_FLOAT);
    dt.u8(0x20);              // little-endian, no padding, mantissa msb implied
    dt.u8(dbl ? 63 : 31);     // sign bit position
    dt.u8(0);
    dt.u32((uint32_t)o.esize);
    dt.u16(0);                // bit offset
    dt.u16(dbl ? 64 : 32);    // precision
    dt.u8(dbl ? 52 : 23);     // exponent location
    dt.u8(dbl ? 11 : 8);      // exponent size
    dt.u8(0);                 // mantissa location
    dt.u8(dbl ? 52 : 23);     // mantissa size
    dt.u32(dbl ? 1023 : 127); // exponent bias
  } else if (o.tclass == T_INT) {
    dt.u8(0x10 | T_INT);
    dt.u8(0x08);              // little-endian, signed
    dt.u8(0);
    dt.u8(0);
    dt.u32((uint32_t)o.esize);
    dt.u16(0);
    dt.u16((unsigned)(8 * o.esize));
  } else {
    dt.u8(0x10 | T_STRING);
    dt.u8(0x01);              // null-padded, ASCII
    dt.u8(0);
    dt.u8(0);
    dt.u32((uint32_t)o.esize);
  }
  m.push_back({M_DTYPE, dt});
  Buf fv;  // Fill Value v3: allocation early, fill never written, default value
  fv.u8(3);
  fv.u8(0x01 | (0x01 << 2));
  m.push_back({M_FILL, fv});
  Buf ly;  // Data Layout v3, contiguous
  ly.u8(3);
  ly.u8(1);
  ly.u64(o.data);
  ly.u64(o.nbytes());
  m.push_back({M_LAYOUT, ly});
  return m;
}

// version 2 object header: "OHDR", version 2, flags (4-byte chunk size),
// chunk size, messages (type, size, flags, data), checksum
static Buf header(const Obj& o) {
  Buf b;
  b.raw("OHDR", 4);
  b.u8(2);
  b.u8(0x02);
  uint32_t chunk = 0;
  auto ms = messages(o);
  for (auto& m : ms) chunk += 4 + (uint32_t)m.second.v.size();
  b.u32(chunk);
  for (auto& m : ms) {
    b.u8((unsigned)m.first);
    b.u16((unsigned)m.second.v.size());
    b.u8(0);
    b.raw(m.second.v.data(), m.second.v.size());
  }
  b.u32(lookup3(b.v.data(), b.v.size(), 0));
  return b;
}

static void collect(Obj& o, std::vector<Obj*>& pre) {
  pre.push_back(&o);
  for (Obj& c : o.kids) collect(c, pre);
}

// Lay out and write the file; false on an I/O error.
bool write_file(const char* path, Obj& root) {
  std::vector<Obj*> objs;
  collect(root, objs);
  // header sizes do not depend on addresses: place headers after the 48-byte
  // superblock in pre-order, then each dataset's raw data (8-byte aligned)
  uint64_t at = 48;
  for (Obj* o : objs) {
    o->ohdr = at;
    at += header(*o).v.size();
  }
  for (Obj* o : objs)
    if (!o->group) {
      at = (at + 7) & ~7ull;
      o->data = at;
      at += o->nbytes();
    }
  const uint64_t eof = at;
  Buf sb;
  sb.raw("\x89HDF\r\n\x1a\n", 8);
  sb.u8(2);  // superblock version
  sb.u8(8);  // size of offsets
  sb.u8(8);  // size of lengths
  sb.u8(0);  // file consistency flags
  sb.u64(0);      // base address
  sb.u64(UNDEF);  // superblock extension address
  sb.u64(eof);    // end of file address
  sb.u64(root.ohdr);
  sb.u32(lookup3(sb.v.data(), sb.v.size(), 0));
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return false;
  bool ok = std::fwrite(sb.v.data(), 1, sb.v.size(), fp) == sb.v.size();
  for (Obj* o : objs) {
    if (!ok) break;
    Buf h = header(*o);
    ok = std::fwrite(h.v.data(), 1, h.v.size(), fp) == h.v.size();
  }
  uint64_t pos = 48;
  for (Obj* o : objs) pos += header(*o).v.size();
  static const uint8_t zeros[8] = {0};
  for (Obj* o : objs) {
    if (!ok) break;
    if (o->group) continue;
    if (o->data > pos) ok = std::fwrite(zeros, 1, o->data - pos, fp) == o->data - pos;
    if (!ok) break;
    if (o->emit) ok = o->emit(fp);
    else ok = o->small.size() == o->nbytes() && std::fwrite(o->small.data(), 1, o->small.size(), fp) == o->small.size();
    pos = o->data + o->nbytes();
  }
  if (std::fclose(fp) != 0) ok = false;
  return ok;
}

// ---- builders ---------------------------------------------------------------
Obj group(const char* name) {
  Obj o;
  o.group = true;
  o.name = name;
  return o;
}
template <typename T> Obj array(const char* name, const T* p, std::vector<uint64_t> dims, TClass tc) {
  Obj o;
  o.group = false;
  o.name = name;
  o.tclass = tc;
  o.esize = (int)sizeof(T);
  o.dims = dims;
  o.small.resize(o.nbytes());
  std::memcpy(o.small.data(), p, o.small.size());
  return o;
}
Obj f64(const char* name, double v) { return array(name, &v, {}, T_FLOAT); }
Obj f64v(const char* name, const std::vector<double>& v) { return array(name, v.data(), {(uint64_t)v.size()}, T_FLOAT); }
Obj i32(const char* name, int v) { return array(name, &v, {}, T_INT); }
Obj str(const char* name, const char* s) {
  Obj o;
  o.group = false;
  o.name = name;
  o.tclass = T_STRING;
  o.esize = (int)std::strlen(s);
  o.small.assign(s, s + o.esize);
  return o;
}

}  // namespace h5w

// ---- the snapshot layout -----------------------------------------------------
// Grid of the padded box: x_i = (i - NG) dx, y likewise, z the layer
// positions (k dz on the uniform grid); the inverse spacings per point are
// 1/dx, 1/dy and, in z, the inverse of dz/dk -- sixth order at the interior
// layers (the metric the kernels use), second-order centred at the ghost
// layers and one-sided at the two outermost ones.  dz is the average
// spacing (z_top - z_bottom) / (nz - 1), L the box lengths n * spacing.
static void grid_group(h5w::Obj& g, const mhd_params* p) {
  const int mx = p->nx + 2 * NG, my = p->ny + 2 * NG, mz = p->nz + 2 * NG;
  std::vector<double> x(mx), y(my), z(mz), dx1(mx, 1.0 / p->dx), dy1(my, 1.0 / p->dy), dz1(mz);
  for (int i = 0; i < mx; ++i) x[i] = (i - NG) * p->dx;
  for (int j = 0; j < my; ++j) y[j] = (j - NG) * p->dy;
  for (int k = 0; k < mz; ++k) z[k] = p->z ? p->z[k] : (k - NG) * p->dz;
  static const double W1[4] = {0.0, 45.0 / 60.0, -9.0 / 60.0, 1.0 / 60.0};
  for (int k = 0; k < mz; ++k) {
    double d;
    if (k >= NG && k < mz - NG) {
      d = 0.0;
      for (int m = 1; m <= 3; ++m) d += W1[m] * (z[k + m] - z[k - m]);
    } else if (k > 0 && k < mz - 1) {
      d = 0.5 * (z[k + 1] - z[k - 1]);
    } else {
      d = k == 0 ? z[1] - z[0] : z[mz - 1] - z[mz - 2];
    }
    dz1[k] = 1.0 / d;
  }
  const double dzm = p->nz > 1 ? (z[mz - 1 - NG] - z[NG]) / (p->nz - 1) : p->dz;
  g.kids.push_back(h5w::f64v("x", x));
  g.kids.push_back(h5w::f64v("y", y));
  g.kids.push_back(h5w::f64v("z", z));
  g.kids.push_back(h5w::f64("dx", p->dx));
  g.kids.push_back(h5w::f64("dy", p->dy));
  g.kids.push_back(h5w::f64("dz", dzm));
  g.kids.push_back(h5w::f64v("dx_1", dx1));
  g.kids.push_back(h5w::f64v("dy_1", dy1));
  g.kids.push_back(h5w::f64v("dz_1", dz1));
  g.kids.push_back(h5w::f64("Lx", p->nx * p->dx));
  g.kids.push_back(h5w::f64("Ly", p->ny * p->dy));
  g.kids.push_back(h5w::f64("Lz", p->nz * dzm));
}

static void settings_group(h5w::Obj& s, const mhd_params* p) {
  s.kids.push_back(h5w::str("precision", p->precision == 64 ? "D" : "S"));
  s.kids.push_back(h5w::i32("nghost", NG));
  s.kids.push_back(h5w::i32("nx", p->nx));
  s.kids.push_back(h5w::i32("ny", p->ny));
  s.kids.push_back(h5w::i32("nz", p->nz));
  s.kids.push_back(h5w::i32("mx", p->nx + 2 * NG));
  s.kids.push_back(h5w::i32("my", p->ny + 2 * NG));
  s.kids.push_back(h5w::i32("mz", p->nz + 2 * NG));
}

static const char* const VAR_NAMES[NF] = {"ax", "ay", "az", "ux", "uy", "uz", "lnrho", "lnTT"};

int h5_write_snapshot(const char* var_path, const char* grid_path, const mhd_params* p, double t,
                      const std::function<bool(int, FILE*)>& field) {
  const uint64_t mx = p->nx + 2 * NG, my = p->ny + 2 * NG, mz = p->nz + 2 * NG;
  if (var_path) {
    h5w::Obj root = h5w::group("");
    root.kids.push_back(h5w::f64("time", t));
    h5w::Obj data = h5w::group("data");
    for (int f = 0; f < NF; ++f) {
      h5w::Obj d;
      d.group = false;
      d.name = VAR_NAMES[f];
      d.tclass = h5w::T_FLOAT;
      d.esize = p->precision == 64 ? 8 : 4;
      d.dims = {mz, my, mx};
      d.emit = [&field, f](FILE* fp) { return field(f, fp); };
      data.kids.push_back(d);
    }
    root.kids.push_back(data);
    h5w::Obj g = h5w::group("grid");
    grid_group(g, p);
    root.kids.push_back(g);
    h5w::Obj s = h5w::group("settings");
    settings_group(s, p);
    root.kids.push_back(s);
    if (!h5w::write_file(var_path, root)) return -1;
  }
  if (grid_path) {
    h5w::Obj root = h5w::group("");
    h5w::Obj g = h5w::group("grid");
    grid_group(g, p);
    root.kids.push_back(g);
    h5w::Obj s = h5w::group("settings");
    settings_group(s, p);
    root.kids.push_back(s);
    if (!h5w::write_file(grid_path, root)) return -1;
  }
  return 0;
}

}  // namespace mhd

extern "C" unsigned int mhd_h5_checksum(const void* data, size_t len) {
  return mhd::h5w::lookup3(data, len, 0);
}
